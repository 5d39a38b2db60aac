// Compile-time-geometry FP32 passes for 90^3 grids.
#define HFX_CT_N 90
#include "hfx_ct.inl"
