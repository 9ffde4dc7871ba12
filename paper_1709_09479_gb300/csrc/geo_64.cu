// Per-map kernels instantiated for 64 x 64 images.
#include "geo_kernels.cuh"

namespace csc {
const GeoOps& geo_ops_64() { return GeoLaunch<GeoCT<64, 64>>::ops(); }
}  // namespace csc
