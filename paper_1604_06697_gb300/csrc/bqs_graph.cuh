// The level loop on the device: a CUDA-graph conditional `while` node whose body is one
// level (pivot, partition, bookkeeping, fills, small-segment and local sorts).  Used
// when a sort is enqueued on a stream that is being captured into a CUDA graph: the
// host then reads nothing back, every kernel takes its level parity from the control
// block, and the last kernel of the body decides whether another level follows.
#pragma once

#include "bqs_kernels.cuh"

namespace bqs {

// First node of the body: the lists this level produces start empty.
static __global__ void k_level_begin(Params P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int q = (P.ctrl->level & 1) ^ 1;
    ListCounts* l = &P.ctrl->lists[q];
    l->large = 0; l->fill = 0; l->large_keys = 0;
    l->small = 0; l->tiny = 0; l->todo = 0; l->local = 0;
  }
}

// Last node of the body: another level runs while the next lists hold work, no error
// was recorded and the level bound (the depth limit plus one halving per key bit, see
// k_pivot) is not exceeded.
static __global__ void k_level_end(Params P, cudaGraphConditionalHandle h, int max_levels) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctrl* c = P.ctrl;
    const int q = (c->level & 1) ^ 1;
    const ListCounts& n = c->lists[q];
    bool more = ((unsigned)n.large | n.small | n.tiny | n.local) != 0u;
    if (c->status != 0) more = false;
    if (more && c->level + 1 > max_levels) {
      c->status = kStatusOverflow;
      more = false;
    }
    c->level += 1;
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

}  // namespace bqs
