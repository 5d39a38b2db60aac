// Compile-time-geometry FP32 passes for 48^3 grids.
#define HFX_CT_N 48
#include "hfx_ct.inl"
