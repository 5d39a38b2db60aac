// Compile-time-geometry FP32 passes for 128^3 grids.
#define HFX_CT_N 128
#include "hfx_ct.inl"
