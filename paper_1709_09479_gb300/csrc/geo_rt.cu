// Per-map kernels instantiated for run-time image sizes.
#include "geo_kernels.cuh"

namespace csc {
const GeoOps& geo_ops_rt() { return GeoLaunch<GeoRT>::ops(); }
}  // namespace csc
