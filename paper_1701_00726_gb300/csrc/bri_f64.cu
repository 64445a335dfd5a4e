// FP64 Brillouin stencil instantiation.
#include "bri_kernel.cuh"

namespace bri {
template int launch_bri_t<double, double2>(const Geom&, double*, const double*, const double2*, const double*,
                                           double, int, int, cudaStream_t, const ShiftDot<double>*, int*);
}  // namespace bri
