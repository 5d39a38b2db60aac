// FP32 instantiation of the exchange passes (FFTs and pair products in FP32).
using Real = float;
#include "hfx_passes.inl"
