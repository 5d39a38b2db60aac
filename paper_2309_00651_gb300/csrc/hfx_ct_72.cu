// Compile-time-geometry FP32 passes for 72^3 grids.
#define HFX_CT_N 72
#include "hfx_ct.inl"
