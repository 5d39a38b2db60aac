// Compile-time-geometry FP32 passes for 96^3 grids.
#define HFX_CT_N 96
#include "hfx_ct.inl"
