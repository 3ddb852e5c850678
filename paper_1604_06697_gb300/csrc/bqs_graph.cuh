// The level loop on the device: a CUDA-graph conditional `while` node whose body is one
// level (pivot, partition, bookkeeping, fills, local partitioning, networks).  Used
// when a sort is enqueued on a stream that is being captured into a CUDA graph: the
// host then reads nothing back, every kernel takes its level parity from the control
// block, and the last kernel of the body decides whether another level follows.
#pragma once

#include "bqs_kernels.cuh"

namespace bqs {

// First kernel of a level: the lists this level produces start empty.  After an error
// (levels enqueued ahead of the host's check) the level's own lists are emptied too,
// so every later kernel of the call finds no work.
static __global__ void k_level_begin(Params P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int p = P.ctrl->level & 1;
    clear_counts(&P.ctrl->lists[p ^ 1]);
    if (P.ctrl->status != 0) clear_counts(&P.ctrl->lists[p]);
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
    bool more = ((unsigned)n.large | n.small | n.tiny | n.local | n.group | n.big) != 0u;
    if (c->status != 0) more = false;
    if (more && c->level + 1 > max_levels) {
      c->status = kStatusOverflow;
      more = false;
    }
    c->level += 1;
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

// Last kernel of one level when the host enqueues levels ahead without reading counts:
// records in a ring indexed by level whether another level has work (bit 0) and
// whether this level partitioned anything (bit 1), adds the level's statistics and
// advances the level.
static __global__ void k_level_step(Params P, int max_levels) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctrl* c = P.ctrl;
    const int lvl = c->level;
    const int p = lvl & 1, q = p ^ 1;
    const ListCounts& cur = c->lists[p];
    const ListCounts& n = c->lists[q];
    if ((unsigned)cur.large != 0u) {
      c->levels_run += 1;
      c->active_total += cur.large_keys;
    }
    c->local_runs += cur.local;
    c->small_runs += cur.small + cur.tiny + cur.group + cur.big;
    bool more = ((unsigned)n.large | n.small | n.tiny | n.local | n.group | n.big) != 0u;
    if (c->status != 0) more = false;
    if (more && lvl + 1 > max_levels) {
      c->status = kStatusOverflow;
      more = false;
    }
    c->more[lvl & 7] = (more ? 1 : 0) | ((unsigned)cur.large != 0u ? 2 : 0);
    c->level = lvl + 1;
  }
}

}  // namespace bqs
