// FP64 instantiation of the exchange passes.
using Real = double;
#include "hfx_passes.inl"
