// Host-side entry points shared between the translation units of librsi.
#pragma once

#include <cuda_runtime.h>

#include "rsi_internal.cuh"

namespace rsi {

// Enqueue the LBVH build (or, with refit, only the bottom-up box pass and the
// treelet) of the meshes described by `ma` into the buffers of `tb` on s.
cudaError_t build_tree(TreeBufs& tb, const MeshArgs& ma, cudaStream_t s, bool refit);

// Raise the box pass's shared-memory limit on the current device (once per
// device; handle creation calls it, so that a first build captured into a
// graph makes no attribute call).
cudaError_t build_prepare();

// Enqueue the 4-wide records of every slot (needs a completed build).
cudaError_t build_nodes4(const TreeBufs& tb, cudaStream_t s);

}  // namespace rsi
