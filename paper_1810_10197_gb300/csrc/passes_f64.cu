// FP64 instantiation of the right-hand-side passes.
#include "passes_impl.cuh"
namespace dns {
template cudaError_t launch_pass<double>(int, const PassArgs&, cudaStream_t);
}
