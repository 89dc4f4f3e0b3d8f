// FP32 instantiation of the right-hand-side passes (transforms and nonlinear term in single
// precision; the P5 epilogue and everything outside the passes stay in double).
#include "passes_impl.cuh"
namespace dns {
template cudaError_t launch_pass<float>(int, const PassArgs&, cudaStream_t);
}
