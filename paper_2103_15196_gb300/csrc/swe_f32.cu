// FP32 state/flux instantiation (FP64 kept for dt, the wet threshold
// semantics, time and volume bookkeeping).  Built with fast-math intrinsics.
#include "swe_launch.cuh"
namespace swe_impl {
SWE_INSTANTIATE(float)
}
