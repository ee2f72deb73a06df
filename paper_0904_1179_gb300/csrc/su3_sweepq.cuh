// su3_sweepq.cuh -- the work queue of the persistent and chained sweeps
// (k_sweep_f32_pair and k_half_sweep_f32_chain in su3_kernels_pair.cu,
// k_sweep_f64 in su3_kernels.cu).
//
// A persistent sweep runs the half-sweeps (mu, parity) of a sweep, in the
// order of the paper's sweep (mu = 0..3, even then odd sites; checkerboard
// updating, Abstract and Sec. 1 of Berg & Wu, arXiv:0904.1179), as tiles of
// one block each.  Tiles are handed out phase by phase from a device counter;
// the tiles of phase q walk the x3 layers of the lattice starting one layer
// further than those of phase q-1, and a tile waits only for the three layers
// of phase q-1 its staples reach (a neighbour x +- nu, x + mu - nu moves x3 by
// at most one).  When a tile of phase q is taken, phase q-1 has handed out
// all its tiles and those layers were among its first three, so in practice
// nothing waits, and the next phase fills the SMs while the previous one
// drains.  Completed layers of phase q-1 imply completed layers of every
// earlier phase around them (each tile waited for its own predecessors before
// it ran), which also keeps a tile from overwriting links that a
// still-running earlier tile reads.  The results are those of the per-phase
// launches bit for bit: the same update of the same links from the same
// inputs.
//
// A block takes its work item from the counter, not from blockIdx, so items
// are handed out in order to blocks that are running: every item a block
// waits for is held by a running block or done, and the lowest item in
// flight never waits, so the order cannot deadlock however many blocks are
// resident.  Every wait is bounded (SweepQueue::wait_ns); when one runs out
// the block sets the status word and every block stops.
//
// Ordering: a block reports its tile with one release reduction by thread 0
// after a block barrier; a waiting block polls the three counts with relaxed
// loads (lanes 0-2 of warp 0), then thread 0 issues one acquire fence and a
// block barrier passes it on -- one acquire per tile, because an acquire also
// drops the SM's L1 lines, which the staging ring of the site-paired kernel
// (cp.async.ca) relies on.
//
// Per direction: four launches per sweep, launch mu holding phases 2 mu and
// 2 mu + 1 (one update variant per launch).  Launches 1-3 are chained to the
// one before by programmatic dependent launch: every block signals
// griddepcontrol.launch_dependents as it starts, so the next launch's blocks
// may be scheduled once all blocks of this one have started, and its first
// phase waits on the layer counts of this one's last phase exactly as the
// phases inside a launch do.  Nothing of a launch waits for a later launch,
// and a later launch's blocks start only when every block of the earlier one
// is running or done, so the chain cannot deadlock either.
//
// Chained half-sweeps: eight launches per sweep, one per phase, chained the
// same way.  A launch holds one phase only, so no tile waits on a tile of its
// own launch; a block's item is its blockIdx (no counter), in the same
// layer-rotated order, and waits only on the launch before, whose blocks have
// all started when this launch's first block does.
#pragma once

#include "su3_device.cuh"
#include "su3_kernels.h"

namespace su3dev {

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Lets the next launch of a chain of per-direction launches be scheduled
// once every block of this one has signalled (or exited).
__device__ __forceinline__ void signal_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A block's work item: phase q (-1: none, the block returns), its tile and
// x3 layer, and its place in the dispatch order of its launch.
struct SweepItem {
  int phase, tile, layer, idx;
};

// Item i of a phase (its place in the dispatch order) -> its x3 layer and
// tile: the phase's tiles walk the layers starting at layer `phase`.
__device__ __forceinline__ void sweep_tile_of(int phase, int i, int tiles_per_layer, int layers, int* layer, int* tile) {
  const int il = i / tiles_per_layer;
  *layer = (il + phase) % layers;
  *tile = *layer * tiles_per_layer + (i - il * tiles_per_layer);
}

// Warp 0 (all 32 lanes) waits, with the bound, for the layers of phase q-1
// that a tile of phase q in `layer` reads, then acquires; false in every lane
// if the sweep stopped.  Phase 0 follows the previous sweep in stream order
// and waits for nothing.
__device__ __forceinline__ bool wait_sweep_layers(const SweepQueue& qa, int phase, int layer, int tiles_per_layer,
                                                  int layers, bool ok) {
  const unsigned* const done = qa.counters + kSweepTickets;
  const int lane = (int)threadIdx.x & 31;
  ok = ok && (lane != 0 || ld_relaxed_s32(qa.status) == 0);
  const bool wait = phase > 0;
  if (wait && lane < 3) {
    // lane k waits for layer l + k - 1 of the previous phase
    const int lk = layer + lane - 1 < 0 ? layers - 1 : (layer + lane - 1 == layers ? 0 : layer + lane - 1);
    const unsigned* cnt = done + (phase - 1) * layers + lk;
    unsigned long long t0 = 0;
    while (ok && ld_relaxed_u32(cnt) < (unsigned)tiles_per_layer) {
      if (t0 == 0) t0 = global_ns();
      if (ld_relaxed_s32(qa.status) != 0) {
        ok = false;
      } else if (global_ns() - t0 > (unsigned long long)qa.wait_ns) {
        atomicCAS(qa.status, 0, kSweepTimeout);
        ok = false;
      } else {
        __nanosleep(64);
      }
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  if (lane == 0 && ok && wait) fence_acquire_gpu();
  return ok;
}

// Warp 0 takes the block's item from counter `ticket` of the queue (the
// launch holds kPhases phases from kFirst on) and waits for the layers of
// phase q-1 it reads; the item lands in *item (shared memory), which the
// block reads after a __syncthreads.
template <int kPhases, int kFirst>
__device__ __forceinline__ void take_sweep_item(const SweepQueue& qa, int ticket, int tiles_per_layer, int layers,
                                                SweepItem* item) {
  if (threadIdx.x >= 32) return;
  const int tiles_per_phase = tiles_per_layer * layers;
  const int lane = (int)threadIdx.x;
  int idx = 0;
  if (lane == 0) idx = (int)atomicAdd(qa.counters + ticket, 1u);
  idx = __shfl_sync(0xffffffffu, idx, 0);
  int phase = -1, tile = 0, layer = 0;
  if (idx < kPhases * tiles_per_phase) {
    phase = kFirst + idx / tiles_per_phase;
    sweep_tile_of(phase, idx - (phase - kFirst) * tiles_per_phase, tiles_per_layer, layers, &layer, &tile);
  }
  const bool ok = wait_sweep_layers(qa, phase, layer, tiles_per_layer, layers, phase >= 0);
  if (lane == 0) *item = SweepItem{ok ? phase : -1, tile, layer, idx};
}

// The same for one half-sweep per launch (the chained half-sweep launches):
// the item is the block's own index, no counter is taken.
__device__ __forceinline__ void own_sweep_item(const SweepQueue& qa, int phase, int tiles_per_layer, int layers,
                                               SweepItem* item) {
  if (threadIdx.x >= 32) return;
  int layer = 0, tile = 0;
  sweep_tile_of(phase, (int)blockIdx.x, tiles_per_layer, layers, &layer, &tile);
  const bool ok = wait_sweep_layers(qa, phase, layer, tiles_per_layer, layers, true);
  if (threadIdx.x == 0) *item = SweepItem{ok ? phase : -1, tile, layer, (int)blockIdx.x};
}

// Reports the block's tile done once every thread's stores are issued.
__device__ __forceinline__ void report_sweep_item(const SweepQueue& qa, int layers, const SweepItem& it) {
  __syncthreads();
  if (threadIdx.x == 0 && it.idx != qa.withhold) red_release_add(qa.counters + kSweepTickets + it.phase * layers + it.layer, 1u);
}

}  // namespace su3dev
