// Double-word instantiation of the right-hand-side passes: transforms, nonlinear term and
// projection in pairs of FP32 values (about 48 significant bits, FP32 instruction rate); the
// P5 epilogue's viscous term and output and everything outside the passes stay in double.
// Each pass is instantiated in its own translation unit (passes_dw_p<k>.cu) so that the
// large kernels compile in parallel.
#include "passes_impl.cuh"
namespace dns {
extern template cudaError_t launch_pass_w<dw, 1>(const PassArgs&, cudaStream_t);
extern template cudaError_t launch_pass_w<dw, 2>(const PassArgs&, cudaStream_t);
extern template cudaError_t launch_pass_w<dw, 3>(const PassArgs&, cudaStream_t);
extern template cudaError_t launch_pass_w<dw, 4>(const PassArgs&, cudaStream_t);
extern template cudaError_t launch_pass_w<dw, 5>(const PassArgs&, cudaStream_t);
template cudaError_t launch_pass<dw>(int, const PassArgs&, cudaStream_t);
}
