// Per-map kernels instantiated for 128 x 128 images.
#include "geo_kernels.cuh"

namespace csc {
const GeoOps& geo_ops_128() { return GeoLaunch<GeoCT<128, 128>>::ops(); }
}  // namespace csc
