// FP32-spinor Brillouin stencil instantiations (FP32 and BF16 link storage).
#include "bri_kernel.cuh"

namespace bri {
template int launch_bri_t<float, float2>(const Geom&, float*, const float*, const float2*, const float*, float, int,
                                         int, cudaStream_t, const ShiftDot<float>*, int*);
template int launch_bri_t<float, __nv_bfloat162>(const Geom&, float*, const float*, const __nv_bfloat162*,
                                                 const float*, float, int, int, cudaStream_t, const ShiftDot<float>*,
                                                 int*);
}  // namespace bri
