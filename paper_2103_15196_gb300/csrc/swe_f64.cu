// FP64 instantiation used for parity with the FP64 CPU oracle.  Built with
// --fmad=false so every operation rounds exactly as written, in the same order
// as the oracle.
#include "swe_launch.cuh"
namespace swe_impl {
SWE_INSTANTIATE(double)
}
