// Compile-time-geometry FP32 passes for 32^3 grids.
#define HFX_CT_N 32
#include "hfx_ct.inl"
