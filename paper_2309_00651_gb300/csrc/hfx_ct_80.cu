// Compile-time-geometry FP32 passes for 80^3 grids.
#define HFX_CT_N 80
#include "hfx_ct.inl"
