// Double-word pass P4 (see passes_dw.cu).
#include "passes_impl.cuh"
namespace dns {
template cudaError_t launch_pass_w<dw, 4>(const PassArgs&, cudaStream_t);
}
