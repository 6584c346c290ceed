// DG1 kernels (placeholder until the Q1 interior-penalty kernels land).
#include "internal.h"
namespace dgls {
cudaError_t dg1_residual(const LaunchCtx&, const DevParams&, const Geo&, const double*, const double*, double, double,
                         int, double*, double*) { return cudaErrorNotSupported; }
template <class S>
cudaError_t dg1_jvp(const LaunchCtx&, const DevParams&, const Geo&, const S*, const S*, double, double, int, double, S*,
                    S*, S*) { return cudaErrorNotSupported; }
template cudaError_t dg1_jvp<double>(const LaunchCtx&, const DevParams&, const Geo&, const double*, const double*, double,
                                     double, int, double, double*, double*, double*);
template cudaError_t dg1_jvp<float>(const LaunchCtx&, const DevParams&, const Geo&, const float*, const float*, double,
                                    double, int, double, float*, float*, float*);
cudaError_t dg1_blocks(const LaunchCtx&, const DevParams&, const Geo&, const double*, double, double, int, double*,
                       double*) { return cudaErrorNotSupported; }
int64_t dg1_face_buffer_len(const DevParams& p) { return p.n_cell; }
}  // namespace dgls
