// mincut_static.cu -- seg_mincut_grid_static: the standalone grid min cut
// without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's allocator regime (a pool that must own every byte), processes
// under a hard device-memory quota set at start-up, or real-time loops where an
// allocation (and the implicit synchronisation it can cause) is forbidden after
// initialisation.  For them this entry point keeps its whole workspace in one
// file-scope device array of fixed size instead of calling cudaMalloc.  The
// array exists on every GPU that loads the library and stays there until the
// process exits.
//
// The scratch array is a host-side stand-in in host code, not a device
// address: its device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and that pointer is what the
// kernel receives.
#include <mutex>
#include <string.h>

#include "seg_internal.cuh"

#define SEG_STATIC_MAX_DEVICES 64

// Workspace bytes the min-cut needs per pixel at the 8-neighbourhood (excess,
// height, sink residual, 8 directed residuals, two flag bytes), plus two bytes
// per pixel for the per-tile words (17 bytes a 32x16 tile: stamp, flag, two
// queue slots and a queue stamp; even a one-column grid, one tile per 16
// pixels, stays under that), the padding of every array to 256 bytes, and the
// status words.
static const size_t kStaticBytes =
    6 * 256 + (size_t)SEG_MINCUT_STATIC_MAX_PIXELS * (3 * 4 + 8 * 4 + 2 + 2) + 8192;

static __device__ __align__(256) unsigned char g_mincut_scratch[kStaticBytes];

static std::mutex g_setup_mu;
static void* g_scratch_addr[SEG_STATIC_MAX_DEVICES];

// Device address of the scratch array on the current device (set up on first use).
static int scratch_on_current_device(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SEG_STATIC_MAX_DEVICES) return SEG_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mincut_scratch) != cudaSuccess || !p) return SEG_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = (char*)g_scratch_addr[dev];
  return SEG_OK;
}

extern "C" int seg_mincut_grid_static(void* stream, int H, int W, int nbr, const int32_t* cs,
                                      const int32_t* ct, const int32_t* ncap, uint8_t* mask,
                                      int64_t* cut, int max_cycles, int* cycles) {
  if (H < 1 || W < 1 || (nbr != 4 && nbr != 8)) return SEG_EINVAL;
  if ((long long)H * W > SEG_MINCUT_STATIC_MAX_PIXELS) return SEG_EINVAL;
  if (!cs || !ct || !ncap || !mask || !cut) return SEG_EINVAL;
  size_t mfb = mf_bytes(H, W, nbr, 1, 0);  // (32x16 tiles: the size bound above assumes them)
  if (mfb + 512 > kStaticBytes) return SEG_EINVAL;
  char* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int grid = 0;
  rc = mf_grid_size(H, W, 0, &grid);
  if (rc) return rc;
  MFWS m;
  mf_bind(m, base, H, W, nbr, 1, 0);
  int* status = (int*)(base + seg_align(mfb));
  // every array the kernel reads before writing starts at zero: status words
  // here, the barrier, round flags and cut accumulator inside mf_launch
  if (cudaMemsetAsync(status, 0, 32, st) != cudaSuccess) return SEG_ECUDA;
  seg_params d;
  seg_default_params(&d);
  MFCall k;
  k.st = st;
  k.grid = grid;
  k.H = H;
  k.W = W;
  k.nbr = nbr;
  k.cs = cs;
  k.ct = ct;
  k.ncap = ncap;
  k.mask_out = mask;
  k.cut_out = (long long*)cut;
  k.status = status;
  k.max_cycles = max_cycles > 0 ? max_cycles : d.max_cycles;
  k.gr_every = d.global_relabel_every;
  k.local_iters = d.local_iters;
  k.timeout_ns = 1000LL * d.barrier_timeout_us;
  k.frontier = d.relabel_frontier;
  rc = mf_launch(m, k, 0);
  if (rc) return rc;
  int hs[4] = {0, 0, 0, 0};
  if (cudaStreamSynchronize(st) != cudaSuccess) return SEG_ECUDA;
  if (cudaMemcpy(hs, status, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess) return SEG_ECUDA;
  if (cycles) *cycles = hs[1];
  return hs[0];
}
