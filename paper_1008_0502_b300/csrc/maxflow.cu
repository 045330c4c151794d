// maxflow.cu -- exact s-t minimum cut of the pixel grid (Sec. 4) on sm_103a.
//
// One persistent cooperative kernel per cut (k_maxflow):
//
//  1. Init: residual capacities of every directed n-link from the undirected
//     capacities; the source arcs are saturated at once and s->v->t flow is
//     cancelled per pixel, so a node starts with excess cs - min(cs, ct) and
//     sink residual ct - min(cs, ct).
//  2. Push-relabel on the "max preflow" (Goldberg-Tarjan first phase): a node is
//     active while it has excess and height < N.  The grid is cut into 32x16
//     tiles coloured by (tile_y mod 2, tile_x mod 2).  In each of the four
//     phases of a cycle only tiles of one colour run; no two of them share a
//     node or an edge, and every node outside a running tile stays fixed, so a
//     phase is a set of independent region discharges (each CTA runs up to
//     local_iters synchronous push / relabel sweeps over its tile in shared
//     memory; pushes into a neighbouring, idle tile go straight to global
//     memory).  A grid barrier separates phases; a colour with no tile that can
//     hold an active node is skipped, barrier included.
//  3. Global relabel every gr_every cycles (one is skipped, never two in a row,
//     after a cycle that left only a little work): exact BFS distances to the sink in
//     the residual graph, computed as a monotone fixpoint (tile-local
//     relaxation in shared memory, rounds of tiles until no value changes);
//     unreachable nodes get height INF and never become active again.
//  4. Stop when no tile of any colour can hold an active node: the preflow is
//     maximum.  The minimal source set is then the
//     residual closure of the nodes that still hold excess (their height is
//     >= N, so they cannot reach t); every minimum cut contains it and it is
//     itself a minimum cut, so the mask is unique.  The cut value is the flow
//     that reached t.
//
// Empty slots of a batch (a.on[fb] == 0) are left out: their rows are treated
// like nodes outside the grid (never read or written), tiles lying wholly in them
// are skipped, and the slot's mask state and warm-start flows keep their values.
// No arc joins two frames, so the other frames' cuts are unchanged.
//
// Every grid barrier waits with a time limit; on expiry the kernel records
// SEG_ETIMEOUT and every CTA returns.  A cycle cap records SEG_ENOTCONVERGED.
#include <string.h>

#include "seg_internal.cuh"

// The tile shape of this copy (seg_params.cut_tile; the build compiles the file
// once per shape, each copy in a namespace of its own).
#ifndef MF_SHAPE
#define MF_SHAPE 0
#endif
#if MF_SHAPE == 0
#define MF_TW 32
#define MF_TH 16
#define MF_NS mf_s32x16
#elif MF_SHAPE == 1
#define MF_TW 32
#define MF_TH 8
#define MF_NS mf_s32x8
#elif MF_SHAPE == 2
#define MF_TW 64
#define MF_TH 8
#define MF_NS mf_s64x8
#else
#error "MF_SHAPE must be 0, 1 or 2"
#endif
#define MF_THREADS (MF_TW * MF_TH)
#define MF_MINB (1024 / MF_THREADS)  // CTAs per SM the kernels are built for (64 registers a thread)

#define MF_HX (MF_TW + 2)
#define MF_HY (MF_TH + 2)
#define MF_HN (MF_HX * MF_HY)
#define MF_ROUND_CAP (1 << 20)  // fixpoint rounds per cut; uniform across CTAs
#ifndef MF_SKIP_GR_TILES
// A cycle with at most this much activity per frame of the stack (tiles left active
// plus colours of tiles pushed into, summed over its phases and CTAs) is not followed
// by a global relabel (640x480 clip: 40 -> cut 96 -> 93 us per frame; 4 and 12 ~ no
// change; 80 and more slower, two-cycle frames then need three; the 64-stream mix at
// default parameters +12 %).
#define MF_SKIP_GR_TILES 40
#endif
#define MF_ON_CACHE 512         // frames whose run flags each CTA keeps in shared memory

namespace MF_NS {

// Directions E W S N SE NW SW NE; the opposite of d is d ^ 1.  The kernel is
// instantiated for 4 and 8 neighbours so every direction loop unrolls and these
// fold to constants.
__device__ __forceinline__ constexpr int mf_dx(int d) {
  return d == 0 ? 1 : d == 1 ? -1 : d == 2 ? 0 : d == 3 ? 0 : d == 4 ? 1 : d == 5 ? -1 : d == 6 ? -1 : 1;
}
__device__ __forceinline__ constexpr int mf_dy(int d) {
  return d == 0 ? 0 : d == 1 ? 0 : d == 2 ? 1 : d == 3 ? -1 : d == 4 ? 1 : d == 5 ? -1 : d == 6 ? 1 : -1;
}
__device__ __forceinline__ constexpr int mf_hoff(int d) { return mf_dy(d) * MF_HX + mf_dx(d); }

struct MFShared {
  int h[MF_HN];  // heights (or BFS distances) with a one-node halo
  int e[MF_THREADS];
  int rt[MF_THREADS];
  int r[8][MF_THREADS];
  unsigned char b[MF_HN];  // residual bitmasks with halo
  unsigned char z[MF_HN];  // reach flags with halo
  int ok;
  unsigned int bar_epoch;  // grid barriers passed in this launch (thread 0)
  unsigned int setmask;  // colours of the tiles this CTA pushed into during a phase
  unsigned int my_tiles;  // tiles this CTA left active during a phase (thread 0)
  unsigned int dmask;    // dirty tiles of a round (mf_dirty_mask)
  long long t_acc[4], t_last;  // phase timing (block 0, thread 0; not in registers)
  unsigned char onf[MF_ON_CACHE];  // the frames' run flags (a.on) when there are at most MF_ON_CACHE
  int on_mode;  // 0: every frame runs, 1: some frame does not (flags in onf), 2: as 1 with the flags in a.on
  unsigned dirs;  // frontier rounds: directions of the neighbour tiles a tile's fixpoint changed
};

__device__ __forceinline__ long long mf_now() { return seg_now(); }

// Grid-wide barrier with a bounded wait (seg_grid_sync); false once this CTA's
// wait or another CTA's has timed out.
__device__ __forceinline__ bool mf_grid_sync(const MFArgs& a, MFShared& s) {
  return seg_grid_sync(a.bar, a.status, a.timeout_ns, &s.ok, &s.bar_epoch);
}

__device__ __forceinline__ unsigned int mf_flag_read(const MFArgs& a, unsigned int epoch) {
  return *(volatile unsigned int*)&a.flags[epoch % 3];
}

// Block-uniform: start a flag round (clears the slot the NEXT round will use).
__device__ __forceinline__ void mf_flag_begin(const MFArgs& a, unsigned int epoch) {
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[(epoch + 1) % 3] = 0u;
}

// Whether frame f of the batch is run.
__device__ __forceinline__ bool mf_frame_on(const MFArgs& a, const MFShared& s, int f) {
  return s.on_mode == 0 || (s.on_mode == 1 ? s.onf[f] : a.on[f]) != 0;
}

// Whether row gy (of the stacked grid) belongs to a frame that is run.
__device__ __forceinline__ bool mf_row_on(const MFArgs& a, const MFShared& s, int gy) {
  return s.on_mode == 0 || mf_frame_on(a, s, gy / a.frame_h);
}

// Block-uniform, for the tile at rows Y0 .. Y0 + MF_TH - 1: bit hy set if halo
// row Y0 - 1 + hy (hy < MF_HY) lies in the grid and in a frame that is run
// (every bit set when every frame runs); *any = some row of the tile itself is
// run (else the tile is skipped).
__device__ __forceinline__ unsigned mf_tile_rows(const MFArgs& a, const MFShared& s, bool all_on, int Y0,
                                                  bool* any) {
  if (all_on) {
    *any = true;
    return ~0u;
  }
  const int g0 = max(Y0 - 1, 0);
  int f = g0 / a.frame_h, next = (f + 1) * a.frame_h;
  bool o = mf_frame_on(a, s, f);
  unsigned m = 0u;
  for (int gy = g0; gy <= min(Y0 + MF_TH, a.H - 1); ++gy) {
    if (gy >= next) {  // (frame_h may be below MF_HY)
      f = gy / a.frame_h;
      next = (f + 1) * a.frame_h;
      o = mf_frame_on(a, s, f);
    }
    if (o) m |= 1u << (gy - (Y0 - 1));
  }
  *any = ((m >> 1) & ((1u << MF_TH) - 1u)) != 0u;
  return m;
}

// Block-uniform: bit i set if tile k0 + i * gridDim.x (i < 32, below ntiles) or
// one of its 8 neighbours changed in a round with epoch >= since (a tile's
// fixpoint can only move when its halo moved).  One read of all the tiles'
// stamps at the start of a round, instead of one dependent read per tile; a
// change made during this round is seen in the next one, which every change
// triggers anyway.
__device__ unsigned mf_dirty_mask(const MFArgs& a, MFShared& s, int k0, int since) {
  if (threadIdx.x == 0) s.dmask = 0u;
  __syncthreads();
  for (int j = threadIdx.x; j < 9 * 32; j += blockDim.x) {
    const int i = j / 9, n = j - 9 * i;
    const int k = k0 + i * (int)gridDim.x;
    if (k < a.ntx * a.nty) {
      const int ty = k / a.ntx, tx = k - ty * a.ntx;
      const int x = tx + n % 3 - 1, y = ty + n / 3 - 1;
      if (x >= 0 && x < a.ntx && y >= 0 && y < a.nty && *(volatile int*)&a.tstamp[y * a.ntx + x] >= since)
        atomicOr(&s.dmask, 1u << i);
    }
  }
  __syncthreads();
  return s.dmask;
}

// ---------------------------------------------------------------- tile frontier
// Block-uniform: bit d set if a node of the tile that changed lies in the halo of
// the neighbour tile in direction d (E W S N SE NW SW NE, as mf_dx / mf_dy): the
// column or row facing it, or the corner node facing a diagonal neighbour.
template <int ND>
__device__ __forceinline__ unsigned mf_rim_dirs(MFShared& s, bool changed, int lx, int ly) {
  unsigned d = 0u;
  if (changed) {
    d = (lx == MF_TW - 1 ? 1u : 0u) | (lx == 0 ? 2u : 0u) | (ly == MF_TH - 1 ? 4u : 0u) | (ly == 0 ? 8u : 0u);
    if (ND == 8)
      d |= ((d & 5u) == 5u ? 16u : 0u) | ((d & 10u) == 10u ? 32u : 0u) | ((d & 6u) == 6u ? 64u : 0u) |
           ((d & 9u) == 9u ? 128u : 0u);
  }
  d = __reduce_or_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && d) atomicOr(&s.dirs, d);
  __syncthreads();  // (also orders the next tile's reuse of shared memory)
  return s.dirs;
}

// Block-uniform (warp 0 works): appends the neighbour tiles in directions dirs to
// the queue of the round with this epoch.  A tile is queued at most once a round:
// the lane whose atomicMax first raises the tile's stamp to the epoch claims it.
// The claiming lanes of the warp take consecutive slots by their rank in the
// ballot, reserved with one atomicAdd on the round's counter (which is also the
// round's termination word: no tile queued, fixpoint reached).
template <int ND>
__device__ __forceinline__ void mf_enqueue(const MFArgs& a, unsigned dirs, int tx, int ty, unsigned epoch,
                                           int ntiles) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  bool claim = false;
  int t = 0;
  if (lane < ND && ((dirs >> lane) & 1u)) {
    const int nx = tx + mf_dx(lane), ny = ty + mf_dy(lane);
    if (nx >= 0 && nx < a.ntx && ny >= 0 && ny < a.nty) {
      t = ny * a.ntx + nx;
      claim = atomicMax(&a.tqs[t], (int)epoch) < (int)epoch;
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, claim);
  if (!m) return;
  unsigned base = 0u;
  if (lane == 0) base = atomicAdd(&a.flags[epoch % 3], (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (claim) a.tq[(size_t)(epoch & 1u) * ntiles + base + __popc(m & ((1u << lane) - 1u))] = t;
}

// ---------------------------------------------------------------- BFS to the sink
// d(u) = 1 if u has residual to t, else 1 + min over residual arcs u->v of d(v):
// relaxed to the local fixpoint with the halo fixed at its current global value.
// Returns whether a node on the tile's rim changed (the only change other tiles
// can see): a round in which no rim changed anywhere is the global fixpoint.
// first: the round that starts a global relabel -- the initial distances (1 on
// nodes with a residual arc to t, INF elsewhere) and the residual bitmasks are
// formed here from rt and r (no separate pass and grid barrier), and every node
// of the tile is written.
// Q: return the directions of the neighbours whose halo changed (mf_rim_dirs)
// instead of whether any rim node changed.
template <int ND, bool Q>
__device__ unsigned mf_tile_bfs(const MFArgs& a, MFShared& s, int tx, int ty, bool first, unsigned rows) {
  const int X0 = tx * MF_TW, Y0 = ty * MF_TH;
  for (int i = threadIdx.x; i < MF_HN; i += blockDim.x) {
    int hy = i / MF_HX, hx = i - hy * MF_HX;
    int gy = Y0 - 1 + hy, gx = X0 - 1 + hx;
    const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W && ((rows >> hy) & 1u);
    const int gg = gy * a.W + gx;
    s.h[i] = !in ? SEG_INF_H : first ? (a.rt[gg] > 0 ? 1 : SEG_INF_H) : a.h[gg];
  }
  const int ly = threadIdx.x / MF_TW, lx = threadIdx.x - ly * MF_TW;
  const int gy = Y0 + ly, gx = X0 + lx;
  const bool valid = gy < a.H && gx < a.W && ((rows >> (ly + 1)) & 1u);
  const int g = gy * a.W + gx;
  const int hi = (ly + 1) * MF_HX + lx + 1;
  unsigned bits = 0u;
  if (valid) {
    if (first) {
#pragma unroll
      for (int d = 0; d < ND; ++d) bits |= (a.r[d * a.N + g] > 0 ? 1u : 0u) << d;
      a.rm[g] = (unsigned char)bits;
    } else {
      bits = a.rm[g];
    }
  }
  __syncthreads();
  if (Q && threadIdx.x == 0) s.dirs = 0u;  // (every thread read the last tile's before the barrier)
  const int h0 = s.h[hi];
  bool any = false;
  for (;;) {
    int ch = 0;
    if (bits) {
      int cur = s.h[hi], nd = cur;
#pragma unroll
      for (int d = 0; d < ND; ++d)
        if ((bits >> d) & 1u) nd = min(nd, s.h[hi + mf_hoff(d)] + 1);
      if (nd < cur) {
        s.h[hi] = nd;
        ch = 1;
      }
    }
    if (!__syncthreads_or(ch)) break;
    any = true;
  }
  if (valid && (any || first)) a.h[g] = s.h[hi];
  // only a change on the tile's rim is seen by other tiles (their halo)
  if (Q) return mf_rim_dirs<ND>(s, valid && s.h[hi] != h0, lx, ly);
  const bool rim = ly == 0 || ly == MF_TH - 1 || lx == 0 || lx == MF_TW - 1;
  return __syncthreads_or(valid && rim && s.h[hi] != h0) != 0;  // (also orders the next tile's reuse)
}

// z(v) = 1 if some residual arc u->v has z(u) = 1 (pull form, halo bitmasks).
// Returns whether a node on the tile's rim changed, as mf_tile_bfs.
// first: the first round -- the seeds are z = 1 where excess remains (no
// separate pass and grid barrier), and every node of the tile is written.  A
// tile with no flag in it or its halo returns at once; otherwise the residual
// bitmasks of the tile and its halo are formed from the residual planes.
template <int ND, bool Q>
__device__ unsigned mf_tile_reach(const MFArgs& a, MFShared& s, int tx, int ty, bool first, unsigned rows) {
  const int X0 = tx * MF_TW, Y0 = ty * MF_TH;
  int seed = 0;
  for (int i = threadIdx.x; i < MF_HN; i += blockDim.x) {
    int hy = i / MF_HX, hx = i - hy * MF_HX;
    int gy = Y0 - 1 + hy, gx = X0 - 1 + hx;
    bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W && ((rows >> hy) & 1u);
    const int gg = gy * a.W + gx;
    const unsigned char zz = !in ? 0 : first ? (a.e[gg] > 0 ? 1 : 0) : a.z[gg];
    s.z[i] = zz;
    seed |= zz;
  }
  const int ly = threadIdx.x / MF_TW, lx = threadIdx.x - ly * MF_TW;
  const int gy = Y0 + ly, gx = X0 + lx;
  const bool valid = gy < a.H && gx < a.W && ((rows >> (ly + 1)) & 1u);
  const int hi = (ly + 1) * MF_HX + lx + 1;
  if (!__syncthreads_or(seed)) {
    // no flag in the tile or its halo: the tile's flags stay 0 this round and its
    // residual planes are not read (most tiles of a frame in the first round)
    if (first && valid) a.z[gy * a.W + gx] = 0;
    return 0u;
  }
  // residual bitmasks of the tile and its halo, from the residual planes
  for (int i = threadIdx.x; i < MF_HN; i += blockDim.x) {
    int hy = i / MF_HX, hx = i - hy * MF_HX;
    int gy2 = Y0 - 1 + hy, gx2 = X0 - 1 + hx;
    bool in = gy2 >= 0 && gy2 < a.H && gx2 >= 0 && gx2 < a.W && ((rows >> hy) & 1u);
    const int gg = gy2 * a.W + gx2;
    unsigned bits = 0u;
    if (in) {
#pragma unroll
      for (int d = 0; d < ND; ++d) bits |= (a.r[d * a.N + gg] > 0 ? 1u : 0u) << d;
    }
    s.b[i] = (unsigned char)bits;
  }
  __syncthreads();
  if (Q && threadIdx.x == 0) s.dirs = 0u;
  const unsigned char z0 = s.z[hi];
  bool any = false;
  for (;;) {
    int ch = 0;
    if (valid && !s.z[hi]) {
      bool hit = false;
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        int nb = hi + mf_hoff(d);
        hit |= s.z[nb] && ((s.b[nb] >> (d ^ 1)) & 1u);
      }
      if (hit) {
        s.z[hi] = 1;
        ch = 1;
      }
    }
    if (!__syncthreads_or(ch)) break;
    any = true;
  }
  if (valid && (any || first)) a.z[gy * a.W + gx] = s.z[hi];
  if (Q) return mf_rim_dirs<ND>(s, valid && s.z[hi] != z0, lx, ly);
  const bool rim = ly == 0 || ly == MF_TH - 1 || lx == 0 || lx == MF_TW - 1;
  return __syncthreads_or(valid && rim && s.z[hi] != z0) != 0;  // (also orders the next tile's reuse)
}

// ---------------------------------------------------------------- region discharge
// Up to local_iters synchronous sweeps over one tile: push along admissible
// arcs (h(u) = h(v) + 1, t has height 0), then relabel every node still active
// to 1 + min over residual arcs.  Returns whether any push or relabel happened.
template <int ND>
__device__ bool mf_discharge(const MFArgs& a, MFShared& s, int tx, int ty, unsigned rows, bool* still_active) {
  const int X0 = tx * MF_TW, Y0 = ty * MF_TH;
  const int N = a.N, W = a.W;
  for (int i = threadIdx.x; i < MF_HN; i += blockDim.x) {
    int hy = i / MF_HX, hx = i - hy * MF_HX;
    int gy = Y0 - 1 + hy, gx = X0 - 1 + hx;
    s.h[i] = (gy >= 0 && gy < a.H && gx >= 0 && gx < W && ((rows >> hy) & 1u)) ? a.h[gy * W + gx] : SEG_INF_H;
  }
  const int tid = threadIdx.x;
  const int ly = tid / MF_TW, lx = tid - ly * MF_TW;
  const int gy = Y0 + ly, gx = X0 + lx;
  const bool valid = gy < a.H && gx < W && ((rows >> (ly + 1)) & 1u);
  const int g = gy * W + gx;
  const int hi = (ly + 1) * MF_HX + lx + 1;
  s.e[tid] = valid ? a.e[g] : 0;
  s.rt[tid] = valid ? a.rt[g] : 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) s.r[d][tid] = valid ? a.r[d * N + g] : 0;
  __syncthreads();
  int work = 0;
  bool remain = true;
  for (int it = 0; it < a.local_iters; ++it) {
    // push
    const int e0 = s.e[tid], hu = s.h[hi];
    if (valid && e0 > 0 && hu < N) {
      int ex = e0;
      if (hu == 1) {
        int rtv = s.rt[tid];
        if (rtv > 0) {
          int dl = min(ex, rtv);
          s.rt[tid] = rtv - dl;
          ex -= dl;
        }
      }
      // the neighbour heights first: they do not change during the push half, but
      // the reverse-arc stores below (s.r[d ^ 1][nt]) would otherwise keep later
      // directions' loads behind them
      int hnv[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) hnv[d] = s.h[hi + mf_hoff(d)];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        if (ex <= 0 || hu != hnv[d] + 1) continue;
        const int rd = s.r[d][tid];
        if (rd <= 0) continue;
        int dl = min(ex, rd);
        s.r[d][tid] = rd - dl;
        ex -= dl;
        int nly = ly + mf_dy(d), nlx = lx + mf_dx(d);
        if (nly >= 0 && nly < MF_TH && nlx >= 0 && nlx < MF_TW) {
          int nt = nly * MF_TW + nlx;
          atomicAdd(&s.e[nt], dl);
          s.r[d ^ 1][nt] += dl;  // only this node writes the reverse arc in this sweep
        } else {
          int gv = g + mf_dy(d) * W + mf_dx(d);
          atomicAdd(&a.e[gv], dl);
          atomicAdd(&a.r[(d ^ 1) * N + gv], dl);
          const int nty = (gy + mf_dy(d)) / MF_TH, ntx = (gx + mf_dx(d)) / MF_TW;
          a.tact[nty * a.ntx + ntx] = 1;
          atomicOr(&s.setmask, 1u << (((nty & 1) << 1) | (ntx & 1)));  // its colour

        }
      }
      if (ex != e0) {
        atomicAdd(&s.e[tid], ex - e0);
        work = 1;
      }
    }
    __syncthreads();
    // relabel
    bool act = false;
    if (valid && s.e[tid] > 0) {
      int cur = s.h[hi];
      if (cur < N) {
        int nh = s.rt[tid] > 0 ? 1 : SEG_INF_H;
#pragma unroll
        for (int d = 0; d < ND; ++d)
          if (s.r[d][tid] > 0) nh = min(nh, s.h[hi + mf_hoff(d)] + 1);
        nh = min(nh, SEG_INF_H);
        if (nh > cur) {
          s.h[hi] = nh;
          work = 1;
          cur = nh;
        }
        act = cur < N;
      }
    }
    if (!__syncthreads_or(act)) {
      remain = false;
      break;
    }
  }
  *still_active = remain;
  // a visit that pushed and relabelled nothing (most tiles of a cycle's first
  // visits: no node with excess) leaves global memory as it was
  const bool changed = __syncthreads_or(work) != 0;
  if (valid && changed) {
    a.e[g] = s.e[tid];
    a.rt[g] = s.rt[tid];
    a.h[g] = s.h[hi];
#pragma unroll
    for (int d = 0; d < ND; ++d) a.r[d * N + g] = s.r[d][tid];
  }
  return changed;  // (the caller's barrier orders the next tile's reuse of shared memory)
}

// ---------------------------------------------------------------- the kernel
__device__ __forceinline__ bool cap_ok(int c) { return c >= 0 && c <= (1 << 24); }

// The whole cut, for one CTA.  SKIP: some frame of the batch is not run (its
// rows are left out); without it every test of the run flags folds away and the
// code is that of a single frame.
template <int ND, bool SKIP, bool Q>
__device__ __forceinline__ void mf_run(const MFArgs& a, MFShared& s) {
  const int N = a.N, W = a.W, H = a.H;
  const int nthr = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntiles = a.ntx * a.nty;
  constexpr bool all_on = !SKIP;

  const long long t_start = mf_now();
  if (threadIdx.x == 0) s.bar_epoch = 0u;  // (read by thread 0 only, in the barriers)
  // ---- 1. init.  Cold: all n-link flows 0.  Warm (a.flow and the frame's warm
  // flag): the previous frame's n-link flows, clamped to the new capacities; a
  // node left with more outflow than its source capacity gets the deficit added
  // to both of its terminal links, which adds the same constant to every cut
  // (minimum cuts unchanged), and the cut value sum(ct - residual to t) with the
  // original ct removes that constant again.
  if (a.init_done) {
    // the terms kernel formed e, rt and r (same arithmetic); each CTA clears the
    // flags of the tiles it takes in the relabel and reach rounds, so no barrier
    // is needed before the first one
    if (threadIdx.x == 0)
      for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        bool any;
        mf_tile_rows(a, s, all_on, (k / a.ntx) * MF_TH, &any);
        a.tstamp[k] = -2;
        if (Q) a.tqs[k] = -1;
        a.tact[k] = any ? 1 : 0;
      }
    __syncthreads();
  } else {
  {  // (restrict, in this block only: the capacity, flow and residual planes never
     // alias, so the unrolled iterations' loads can be issued ahead of the stores)
  const int32_t* __restrict__ in_cs = a.cs;
  const int32_t* __restrict__ in_ct = a.ct;
  const int32_t* __restrict__ ncap = a.ncap;
  const int* __restrict__ flow_in = a.flow;
  int* __restrict__ r_out = a.r;
#pragma unroll 2
  for (int u = gtid; u < N; u += nthr) {
    int y = u / W, x = u - y * W;
    if (SKIP && !mf_row_on(a, s, y)) continue;
    int cs = in_cs[u], ct = in_ct[u];
    bool bad = !cap_ok(cs) || !cap_ok(ct);
    const bool up = y > 0 && (!SKIP || mf_row_on(a, s, y - 1));  // (an empty slot's rows above: outside)
    const int cE = x + 1 < W ? ncap[u] : 0;
    const int cW = x > 0 ? ncap[u - 1] : 0;
    const int cS = y + 1 < H ? ncap[N + u] : 0;
    const int cN = up ? ncap[N + u - W] : 0;
    bad |= !cap_ok(cE) || !cap_ok(cS);
    const bool warm = a.flow != nullptr && a.warm[y / a.frame_h];
    auto clampf = [](int f, int c) { return f > c ? c : (f < -c ? -c : f); };
    // forward flows leave u (E, S, SE, SW); backward ones (W, N, NW, NE) enter u
    const int fE = warm && x + 1 < W ? clampf(flow_in[u], cE) : 0;
    const int fW = warm && x > 0 ? clampf(flow_in[u - 1], cW) : 0;
    const int fS = warm && y + 1 < H ? clampf(flow_in[N + u], cS) : 0;
    const int fN = warm && up ? clampf(flow_in[N + u - W], cN) : 0;
    int net_out = fE - fW + fS - fN;
    r_out[0 * N + u] = cE - fE;
    r_out[1 * N + u] = cW + fW;
    r_out[2 * N + u] = cS - fS;
    r_out[3 * N + u] = cN + fN;
    if (ND == 8) {
      const int cSE = (x + 1 < W && y + 1 < H) ? ncap[2 * N + u] : 0;
      const int cNW = (x > 0 && up) ? ncap[2 * N + u - W - 1] : 0;
      const int cSW = (x > 0 && y + 1 < H) ? ncap[3 * N + u] : 0;
      const int cNE = (x + 1 < W && up) ? ncap[3 * N + u - W + 1] : 0;
      bad |= !cap_ok(cSE) || !cap_ok(cSW);
      const int fSE = warm && x + 1 < W && y + 1 < H ? clampf(flow_in[2 * N + u], cSE) : 0;
      const int fNW = warm && x > 0 && up ? clampf(flow_in[2 * N + u - W - 1], cNW) : 0;
      const int fSW = warm && x > 0 && y + 1 < H ? clampf(flow_in[3 * N + u], cSW) : 0;
      const int fNE = warm && x + 1 < W && up ? clampf(flow_in[3 * N + u - W + 1], cNE) : 0;
      net_out += fSE - fNW + fSW - fNE;
      r_out[4 * N + u] = cSE - fSE;
      r_out[5 * N + u] = cNW + fNW;
      r_out[6 * N + u] = cSW - fSW;
      r_out[7 * N + u] = cNE + fNE;
    }
    int e0 = cs - net_out, cte = ct;
    if (e0 < 0) {  // deficit
      cte = ct - e0;
      e0 = 0;
    }
    const int m = min(e0, cte);
    a.e[u] = e0 - m;
    a.rt[u] = cte - m;
    if (bad) atomicCAS(&a.status[0], 0, SEG_ECAPACITY);
  }
  }
  for (int t = gtid; t < ntiles; t += nthr) {
    bool any;
    mf_tile_rows(a, s, all_on, (t / a.ntx) * MF_TH, &any);
    a.tstamp[t] = -2;
    if (Q) a.tqs[t] = -1;
    a.tact[t] = any ? 1 : 0;
  }
  if (!mf_grid_sync(a, s)) return;
  if (*(volatile int*)&a.status[0] == SEG_ECAPACITY) return;
  }

  unsigned int epoch = 0;
  int cycle = 0, n_gr = 0, n_rounds = 0;
  bool converged = false;
  // phase timing on one thread (the grid moves in lock-step between barriers):
  // [0] init, [1] global relabels, [2] discharge cycles, [3] final reach + mask
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) s.t_acc[k] = 0;
    s.t_last = t_start;
  }
  auto lap = [&](int slot) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      long long t = mf_now();
      s.t_acc[slot] += t - s.t_last;
      s.t_last = t;
    }
  };
  lap(0);
  // Phase scheduling.  Bit c of flag: some tile of colour c may hold an active node.
  // Every CTA keeps the same copy, updated only from the word the phase's CTAs
  // OR together before its barrier (bit c': a push entered a tile of colour c';
  // bit 4: a tile of the discharged colour is still active), so skipping a
  // colour -- and its barrier -- is decided identically everywhere.  The
  // preflow is maximum once no colour is flagged.  A global relabel runs first
  // and then after every 4 * gr_every executed phases.
  unsigned int flag = 15u;
  int color = 0, executed = 0, since_gr = 0;
  bool relabel = true;
  // activity since the last relabel (tiles left active, colours pushed into, summed
  // over the CTAs and phases), the same in every CTA; bit 31: the last relabel was skipped
  unsigned act_since_gr = 0u;
  for (;;) {
    int tries = 0;
    while (tries < 4 && !((flag >> color) & 1u)) {
      color = (color + 1) & 3;
      ++tries;
    }
    if (tries == 4) {
      converged = true;
      break;
    }
    if (executed >= 4 * a.max_cycles) break;
    // ---- 3. global relabel (a cycle that left only a few tiles to work on goes on
    // without one, at most once in a row: the labels stay valid, and a relabel of
    // every tile would cost more than the few visits it could shorten)
    if (!relabel && since_gr >= 4 * a.gr_every && act_since_gr <= (unsigned)(MF_SKIP_GR_TILES * a.nframes)) {
      since_gr = 0;
      act_since_gr = 0x80000000u;
    }
    if (relabel || since_gr >= 4 * a.gr_every) {
      relabel = false;
      since_gr = 0;
      act_since_gr = 0u;
      for (int rnd = 0;; ++rnd) {
        const bool first = rnd == 0;
        mf_flag_begin(a, epoch);
        bool ch = false;
        if (Q && rnd >= 2) {  // the tiles the previous round queued, spread over the CTAs
          const int cnt = (int)mf_flag_read(a, epoch - 1);
          const int* q = a.tq + (size_t)((epoch - 1) & 1u) * ntiles;
          for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
            const int k = q[i], tx = k % a.ntx, ty = k / a.ntx;
            bool any;
            const unsigned rows = mf_tile_rows(a, s, all_on, ty * MF_TH, &any);
            if (!any) continue;
            const unsigned d = mf_tile_bfs<ND, true>(a, s, tx, ty, false, rows);
            if (d) mf_enqueue<ND>(a, d, tx, ty, epoch, ntiles);
          }
        } else {
          unsigned dm = 0u;
          for (int k = blockIdx.x, i = 0; k < ntiles; k += gridDim.x, ++i) {
            int tx = k % a.ntx, ty = k / a.ntx;
            if (!first) {
              if ((i & 31) == 0) dm = mf_dirty_mask(a, s, k, (int)epoch - 1);
              if (!((dm >> (i & 31)) & 1u)) continue;
            }
            bool any;
            const unsigned rows = mf_tile_rows(a, s, all_on, ty * MF_TH, &any);
            if (!any) continue;
            const unsigned d = mf_tile_bfs<ND, Q>(a, s, tx, ty, first, rows);
            if (!d) continue;
            if (Q && !first) {  // (claims start after a barrier: every stamp was reset by then)
              mf_enqueue<ND>(a, d, tx, ty, epoch, ntiles);
            } else {
              ch = true;
              if (threadIdx.x == 0) a.tstamp[k] = (int)epoch;
            }
          }
        }
        if (ch && threadIdx.x == 0) atomicAdd(&a.flags[epoch % 3], 1u);
        if (!mf_grid_sync(a, s)) return;
        unsigned int f = mf_flag_read(a, epoch);
        ++epoch;
        ++n_rounds;
        if (f == 0u) break;
        if (n_rounds >= MF_ROUND_CAP) {
          if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.status[0], 0, SEG_ENOTCONVERGED);
          return;
        }
      }
      ++n_gr;
      lap(1);
    }
    // ---- 2. one colour phase
    {
      mf_flag_begin(a, epoch);
      if (threadIdx.x == 0) {
        s.setmask = 0u;
        s.my_tiles = 0u;
      }
      __syncthreads();
      const int cy = color >> 1, cx = color & 1;
      const int ntx_c = (a.ntx - cx + 1) / 2, nty_c = (a.nty - cy + 1) / 2;
      const int ntc = ntx_c * nty_c;
      bool any_remain = false;
      for (int k = blockIdx.x; k < ntc; k += gridDim.x) {
        const int tx = 2 * (k % ntx_c) + cx, ty = 2 * (k / ntx_c) + cy, t = ty * a.ntx + tx;
        if (!*(volatile unsigned char*)&a.tact[t]) continue;  // no active node can be in it
        bool remain, any;
        const unsigned rows = mf_tile_rows(a, s, all_on, ty * MF_TH, &any);
        mf_discharge<ND>(a, s, tx, ty, rows, &remain);
        __syncthreads();
        if (threadIdx.x == 0) {
          a.tact[t] = remain ? 1 : 0;
          s.my_tiles += remain ? 1u : 0u;
        }
        any_remain |= remain;
      }
      __syncthreads();
      const unsigned int bits = s.setmask | (any_remain ? 16u : 0u);
      if (threadIdx.x == 0) {
        if (bits) atomicOr(&a.flags[epoch % 3], bits);
        // bits 8 and up: this CTA's activity (tiles left active, colours of tiles pushed into),
        // added beside the OR-ed bits without touching them
        const unsigned act = s.my_tiles + __popc(s.setmask);
        if (act) atomicAdd(&a.flags[epoch % 3], min(act, 0xffffu) << 8);
      }
      if (!mf_grid_sync(a, s)) return;
      const unsigned int f = mf_flag_read(a, epoch);
      act_since_gr += f >> 8;
      ++epoch;
      flag = ((flag | f) & 15u & ~(1u << color)) | (((f >> 4) & 1u) << color);
      color = (color + 1) & 3;
      ++executed;
      ++since_gr;
      cycle = (executed + 3) / 4;
    }
    lap(2);
  }

  // ---- 4. minimal source set and cut value (the flow that reached t, per frame
  // of a stacked batch: rows fb*frame_h .. fb*frame_h + frame_h - 1)
  {
    const int nf = a.frame_h * W;  // nodes per frame
    for (int fb = 0; fb < a.nframes; ++fb) {
      if (SKIP && !mf_frame_on(a, s, fb)) continue;
      long long flow_t = 0;
      for (int u = fb * nf + gtid; u < (fb + 1) * nf; u += nthr) flow_t += (long long)a.ct[u] - a.rt[u];
      for (int o = 16; o > 0; o >>= 1) flow_t += __shfl_xor_sync(0xffffffffu, flow_t, o);
      if ((threadIdx.x & 31) == 0 && flow_t != 0) atomicAdd(&a.cut_acc[fb], (unsigned long long)flow_t);
    }
  }
  for (int rnd = 0;; ++rnd) {
    const bool first = rnd == 0;
    mf_flag_begin(a, epoch);
    bool ch = false;
    if (Q && rnd >= 2) {
      const int cnt = (int)mf_flag_read(a, epoch - 1);
      const int* q = a.tq + (size_t)((epoch - 1) & 1u) * ntiles;
      for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        const int k = q[i], tx = k % a.ntx, ty = k / a.ntx;
        bool any;
        const unsigned rows = mf_tile_rows(a, s, all_on, ty * MF_TH, &any);
        if (!any) continue;
        const unsigned d = mf_tile_reach<ND, true>(a, s, tx, ty, false, rows);
        if (d) mf_enqueue<ND>(a, d, tx, ty, epoch, ntiles);
      }
    } else {
      unsigned dm = 0u;
      for (int k = blockIdx.x, i = 0; k < ntiles; k += gridDim.x, ++i) {
        int tx = k % a.ntx, ty = k / a.ntx;
        if (!first) {
          if ((i & 31) == 0) dm = mf_dirty_mask(a, s, k, (int)epoch - 1);
          if (!((dm >> (i & 31)) & 1u)) continue;
        }
        bool any;
        const unsigned rows = mf_tile_rows(a, s, all_on, ty * MF_TH, &any);
        if (!any) continue;
        const unsigned d = mf_tile_reach<ND, Q>(a, s, tx, ty, first, rows);
        if (!d) continue;
        if (Q && !first) {
          mf_enqueue<ND>(a, d, tx, ty, epoch, ntiles);
        } else {
          ch = true;
          if (threadIdx.x == 0) a.tstamp[k] = (int)epoch;
        }
      }
    }
    if (ch && threadIdx.x == 0) atomicAdd(&a.flags[epoch % 3], 1u);
    if (!mf_grid_sync(a, s)) return;
    unsigned int f = mf_flag_read(a, epoch);
    ++epoch;
    ++n_rounds;
    if (f == 0u) break;
    if (n_rounds >= MF_ROUND_CAP) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.status[0], 0, SEG_ENOTCONVERGED);
      return;
    }
  }
  uint8_t* mask_out = a.mask_out ? a.mask_out : a.io->mask;
  for (int u = gtid; u < N; u += nthr) {
    if (!all_on && !mf_row_on(a, s, u / W)) continue;  // (an empty slot's state is kept)
    uint8_t v = a.z[u];
    mask_out[u] = v;
    if (a.mask_state) a.mask_state[u] = v;
    if (a.flow) {  // n-link flows of this cut, the next frame's warm start
      const int y = u / W, x = u - y * W;
      a.flow[u] = x + 1 < W ? a.ncap[u] - a.r[0 * N + u] : 0;
      a.flow[N + u] = y + 1 < H ? a.ncap[N + u] - a.r[2 * N + u] : 0;
      if (ND == 8) {
        a.flow[2 * N + u] = (x + 1 < W && y + 1 < H) ? a.ncap[2 * N + u] - a.r[4 * N + u] : 0;
        a.flow[3 * N + u] = (x > 0 && y + 1 < H) ? a.ncap[3 * N + u] - a.r[6 * N + u] : 0;
      }
    }
  }
  if (a.flow && blockIdx.x == 0)
    for (int fb = threadIdx.x; fb < a.nframes; fb += blockDim.x)
      if (!SKIP || mf_frame_on(a, s, fb)) a.warm[fb] = 1;
  long long* cut_out = a.cut_out ? a.cut_out : (a.io ? a.io->cut : nullptr);
  if (cut_out && blockIdx.x == 0)
    for (int fb = threadIdx.x; fb < a.nframes; fb += blockDim.x)
      cut_out[fb] = (long long)*(volatile unsigned long long*)&a.cut_acc[fb];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!converged) atomicCAS(&a.status[0], 0, SEG_ENOTCONVERGED);
    a.status[1] = cycle;
    a.status[2] = n_gr;
    a.status[3] = n_rounds;
    lap(3);
    for (int k = 0; k < 4; ++k) a.status[4 + k] = (int)(s.t_acc[k] / 100);  // units of 0.1 us
  }
}

// One frame: only the schedule varies.
template <int ND>
__global__ void __launch_bounds__(MF_THREADS, MF_MINB) k_maxflow(MFArgs a) {
  __shared__ MFShared s;
  if (a.frontier)
    mf_run<ND, false, true>(a, s);
  else
    mf_run<ND, false, false>(a, s);
}

// A stack of frames (a batch context): empty slots are left out when a.on marks
// some.  A kernel of its own, so that the single-frame code keeps its own
// register allocation.
template <int ND>
__global__ void __launch_bounds__(MF_THREADS, MF_MINB) k_maxflow_batch(MFArgs a) {
  __shared__ MFShared s;
  int off = 0;
  if (a.on) {  // its frames' run flags, read once per CTA
    for (int f = threadIdx.x; f < a.nframes; f += blockDim.x) {
      const unsigned char v = a.on[f];
      if (f < MF_ON_CACHE) s.onf[f] = v;
      off |= v == 0;
    }
    off = __syncthreads_or(off);
    if (threadIdx.x == 0) s.on_mode = !off ? 0 : (a.nframes <= MF_ON_CACHE ? 1 : 2);
    __syncthreads();
  }
  if (off) {
    if (a.frontier) mf_run<ND, true, true>(a, s);
    else mf_run<ND, true, false>(a, s);
  } else {
    if (a.frontier) mf_run<ND, false, true>(a, s);
    else mf_run<ND, false, false>(a, s);
  }
}

// ---------------------------------------------------------------- host side
size_t bytes(int H, int W, int ndir, int nframes) {
  size_t N = (size_t)H * W;
  size_t nt = (size_t)((W + MF_TW - 1) / MF_TW) * ((H + MF_TH - 1) / MF_TH);
  return seg_align(N * 4) * 3 + seg_align(N * 4 * ndir) + seg_align(N) * 2 + seg_align(8 * nframes) +
         seg_align(16) + seg_align(nt * 4) + seg_align(nt) + seg_align(sizeof(GridBar)) + seg_align(nt * 8) +
         seg_align(nt * 4);
}

void bind(MFWS& m, char* base, int H, int W, int ndir, int nframes) {
  size_t N = (size_t)H * W, off = 0;
  auto take = [&](size_t b) {
    char* p = base + off;
    off += seg_align(b);
    return p;
  };
  m.e = (int*)take(N * 4);
  m.h = (int*)take(N * 4);
  m.rt = (int*)take(N * 4);
  m.r = (int*)take(N * 4 * ndir);
  m.rm = (unsigned char*)take(N);
  m.z = (unsigned char*)take(N);
  m.cut_acc = (unsigned long long*)take(8 * nframes);
  m.nframes = nframes;
  m.flags = (unsigned int*)take(16);
  size_t nt = (size_t)((W + MF_TW - 1) / MF_TW) * ((H + MF_TH - 1) / MF_TH);
  m.tstamp = (int*)take(nt * 4);
  m.tact = (unsigned char*)take(nt);
  m.bar = (GridBar*)take(sizeof(GridBar));
  m.tq = (int*)take(nt * 8);
  m.tqs = (int*)take(nt * 4);
}

int grid_size(int H, int W, int* grid) {
  int dev, nsm, per_sm = 0, coop = 0;
  SEG_CUDA_TRY(cudaGetDevice(&dev));
  SEG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SEG_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return SEG_ECUDA;
  SEG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_maxflow<8>, MF_THREADS, 0));
  const void* others[3] = {(const void*)k_maxflow<4>, (const void*)k_maxflow_batch<8>,
                           (const void*)k_maxflow_batch<4>};
  for (const void* k : others) {
    int n = 0;
    SEG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, MF_THREADS, 0));
    per_sm = n < per_sm ? n : per_sm;
  }
  if (per_sm < 1) return SEG_ECUDA;
  const int ntx = (W + MF_TW - 1) / MF_TW, nty = (H + MF_TH - 1) / MF_TH;
  const int ntiles = ntx * nty, ntc = ((ntx + 1) / 2) * ((nty + 1) / 2);  // tiles; of the largest colour
  // A phase walks its colour's tiles and a relabel / reach round all tiles, CTA
  // k taking tiles k, k + grid, ..; the step lasts as long as the CTA with the
  // most tiles.  With every co-resident CTA those counts are at their minimum
  // (rp per phase, ra per round); the grid is the fewest CTAs that still reach
  // both (fewer arrivals per barrier, and idle SMs for concurrent work), e.g.
  // 640 x 480 in 32x16 tiles: 150 tiles per colour, 600 in all -> 200 CTAs (1
  // and 3 tiles).
  const int gmax = per_sm * nsm;
  const int rp = (ntc + gmax - 1) / gmax, ra = (ntiles + gmax - 1) / gmax;
  const int gp = (ntc + rp - 1) / rp, ga = (ntiles + ra - 1) / ra;
  *grid = gp > ga ? gp : ga;
  return SEG_OK;
}

int launch(const MFWS& m, const MFCall& c) {
  if (c.H % m.nframes) return SEG_EINVAL;
  MFArgs a;
  memset(&a, 0, sizeof(a));
  a.on = c.on;
  a.frontier = c.frontier ? 1 : 0;
  a.tq = m.tq;
  a.tqs = m.tqs;
  a.flow = c.flow;
  a.warm = c.warm;
  a.nframes = m.nframes;
  a.frame_h = c.H / m.nframes;
  a.H = c.H;
  a.W = c.W;
  a.N = c.H * c.W;
  a.ndir = c.nbr;
  a.ntx = (c.W + MF_TW - 1) / MF_TW;
  a.nty = (c.H + MF_TH - 1) / MF_TH;
  a.cs = c.cs;
  a.ct = c.ct;
  a.ncap = c.ncap;
  a.e = m.e;
  a.h = m.h;
  a.rt = m.rt;
  a.r = m.r;
  a.rm = m.rm;
  a.z = m.z;
  a.mask_out = c.mask_out;
  a.mask_state = c.mask_state;
  a.cut_out = c.cut_out;
  a.io = c.io;
  a.cut_acc = m.cut_acc;
  a.flags = m.flags;
  a.tstamp = m.tstamp;
  a.tact = m.tact;
  a.bar = m.bar;
  a.status = c.status;
  a.max_cycles = c.max_cycles;
  a.gr_every = c.gr_every < 1 ? 1 : c.gr_every;
  a.local_iters = c.local_iters < 1 ? 1 : c.local_iters;
  a.timeout_ns = c.timeout_ns;
  a.init_done = c.init_done ? 1 : 0;
  if (!c.words_zeroed) {  // (else the caller's frame-start kernel has zeroed them)
    SEG_CUDA_TRY(cudaMemsetAsync(m.cut_acc, 0, 8 * m.nframes, c.st));
    SEG_CUDA_TRY(cudaMemsetAsync(m.flags, 0, 16, c.st));
    SEG_CUDA_TRY(cudaMemsetAsync(m.bar, 0, sizeof(GridBar), c.st));
  }
  void* args[] = {&a};
  const void* fn = m.nframes > 1
                       ? (c.nbr == 8 ? (const void*)k_maxflow_batch<8> : (const void*)k_maxflow_batch<4>)
                       : (c.nbr == 8 ? (const void*)k_maxflow<8> : (const void*)k_maxflow<4>);
  SEG_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(c.grid), dim3(MF_THREADS), args, 0, c.st));
  return SEG_OK;
}

}  // namespace MF_NS
