// Segmentation on the GPU (moc_track.cu): the Walker that generate_tracks calls to run the
// half-edge walk of every ray on the device.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "moc_geom.h"

namespace moc {

struct DeviceWalkCtx {
  int device;
  cudaStream_t stream;
  double walk_ms;  // device time of the count and fill passes of the last walk
};

// Walker::run for a DeviceWalkCtx: uploads the mesh and the rays, counts tracks and segments per
// ray, fills them at prefix-sum offsets and copies the result to `out` (ray order).
int device_walk(void *ctx, const Geometry &g, const RayBatch &rays, WalkResult &out, std::string &err);

}  // namespace moc
