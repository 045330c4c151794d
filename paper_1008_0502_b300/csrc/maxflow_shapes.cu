// maxflow_shapes.cu -- the min cut's entry points for every tile shape.
//
// maxflow.cu is compiled once per tile shape (MF_SHAPE = 0, 1, 2: 32x16, 32x8
// and 64x8 nodes), each copy in a namespace of its own; these functions pick
// the copy of seg_params.cut_tile.  The workspace layout depends on the shape
// (one stamp, flag and queue slot per tile), so a context keeps one shape.
#include "seg_internal.cuh"

#define MF_DECLARE(ns)                                                 \
  namespace ns {                                                       \
  size_t bytes(int H, int W, int ndir, int nframes);                   \
  void bind(MFWS& m, char* base, int H, int W, int ndir, int nframes); \
  int grid_size(int H, int W, int* grid);                              \
  int launch(const MFWS& m, const MFCall& c);                          \
  }
MF_DECLARE(mf_s32x16)
MF_DECLARE(mf_s32x8)
MF_DECLARE(mf_s64x8)

size_t mf_bytes(int H, int W, int ndir, int nframes, int shape) {
  return shape == 1   ? mf_s32x8::bytes(H, W, ndir, nframes)
         : shape == 2 ? mf_s64x8::bytes(H, W, ndir, nframes)
                      : mf_s32x16::bytes(H, W, ndir, nframes);
}

void mf_bind(MFWS& m, char* base, int H, int W, int ndir, int nframes, int shape) {
  if (shape == 1)
    mf_s32x8::bind(m, base, H, W, ndir, nframes);
  else if (shape == 2)
    mf_s64x8::bind(m, base, H, W, ndir, nframes);
  else
    mf_s32x16::bind(m, base, H, W, ndir, nframes);
}

int mf_grid_size(int H, int W, int shape, int* grid) {
  return shape == 1   ? mf_s32x8::grid_size(H, W, grid)
         : shape == 2 ? mf_s64x8::grid_size(H, W, grid)
                      : mf_s32x16::grid_size(H, W, grid);
}

int mf_launch(const MFWS& m, const MFCall& c, int shape) {
  if (shape < 0 || shape >= SEG_CUT_TILES) return SEG_EINVAL;
  return shape == 1 ? mf_s32x8::launch(m, c) : shape == 2 ? mf_s64x8::launch(m, c) : mf_s32x16::launch(m, c);
}
