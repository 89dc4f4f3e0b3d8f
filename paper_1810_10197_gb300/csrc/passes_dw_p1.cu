// Double-word pass P1 (see passes_dw.cu).
#include "passes_impl.cuh"
namespace dns {
template cudaError_t launch_pass_w<dw, 1>(const PassArgs&, cudaStream_t);
}
