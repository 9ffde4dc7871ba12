// Per-map kernels instantiated for 100 x 100 images.
#include "geo_kernels.cuh"

namespace csc {
const GeoOps& geo_ops_100() { return GeoLaunch<GeoCT<100, 100>>::ops(); }
}  // namespace csc
