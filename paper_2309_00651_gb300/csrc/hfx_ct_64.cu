// Compile-time-geometry FP32 passes for 64^3 grids.
#define HFX_CT_N 64
#include "hfx_ct.inl"
