// Fused COCG iteration: declarations.
#pragma once
#include "cocg.cuh"

namespace rpa {


template <typename T>
struct FusedBufs {
  cpx<T>* p_in;            // p_{k-1}
  cpx<T>* p_out;           // p_k
  cpx<T>* cp;              // projector coefficients of p_k (gamma dV chi^T p), nsys x ng x 4
  cpx<T>* cr;              // projector sums of r, accumulated by the update kernel
  const int* tile_roff;    // per 1-D tile: offsets into the range list
  const int* tile_ranges;  // (group, first entry, end entry) of group-major entries in a tile
  int ntiles_xy, nzchunk, zchunk, tiles1d, first;
  int nact;                // launched systems: the first nact entries of CocgView::list
  int row_ty;              // 0: 32 x 8 column tiles; > 0: row tiles of this height (nx <= 64);
                           // kTileX2: 64 x 8 tiles, two x points per thread (FP32, nx even);
                           // band_code(h): bands of h full rows, two points per thread;
                           // kTileX2Packed: two-point kernel on packed full rows
  int band_ty;             // rows of a band (band tiling only)
};

constexpr int kTileX2 = -2;
// the two-point tiles with the z window in a shared-memory ring (see cocg_x2.cu): one centre
// plane buffer (three blocks per SM) or two
constexpr int kTileX2Ring1 = -3, kTileX2Ring2 = -4;
inline bool is_x2(int code) {
  return code == kTileX2 || code == kTileX2Ring1 || code == kTileX2Ring2;
}
cudaError_t launch_dirmatvec_x2_prepare();
// two-point kernel on packed full rows (see cocg_x2p.cu): FP32, R = 6, even nx in [26, 64]
constexpr int kTileX2Packed = -6;
bool x2p_tile_fits(int nx, int R);
int x2p_tiles_xy(int nx, int ny);
cudaError_t launch_dirmatvec_x2p(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                 cudaStream_t s);
// tiling codes of the band kernel: -100 - h for bands of h rows
constexpr int kTileBandBase = -100;
inline int band_code(int ty) { return kTileBandBase - ty; }
inline bool is_band(int code) { return code < kTileBandBase; }
inline int band_rows(int code) { return kTileBandBase - code; }
// band kernel (FP32, nx even and <= 64, h | ny): whether bands of ty rows fit, the heights
// worth timing, its one-time function attributes (call before a stream capture), the launch
bool band_tile_fits(int nx, int ny, int R, int ty, int ngroup);
int band_candidates(int nx, int ny, int R, int ngroup, int* out, int maxn);
cudaError_t launch_dirmatvec_band_prepare();
cudaError_t launch_dirmatvec_band(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                  cudaStream_t s);
bool x2_tile_fits(int nx, int R);
int x2_tiles_xy(int nx, int ny);
cudaError_t launch_dirmatvec_x2(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                cudaStream_t s);

// whether full-row tiles of height ty can run on an nx x ny plane with stencil radius R
template <typename T>
bool row_tile_fits(int nx, int ny, int R, int ty);
// row-tile heights worth timing for this grid (none when nx > 64); returns the count
template <typename T>
int row_candidates(int nx, int ny, int R, int ngroup, int* out, int maxn);
template <typename T>
cudaError_t launch_dirmatvec_rows(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s);
// one-time function attributes of the row kernels (call before a stream capture)
template <typename T>
cudaError_t launch_dirmatvec_rows_prepare();

// the direction + H-apply kernel alone (used by the tile autotuner)
template <typename T>
cudaError_t launch_dirmatvec_only(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s);

template <typename T>
cudaError_t fused_iteration(const CocgView<T>& cv, const FusedBufs<T>& fb, double tol, int maxit,
                            cudaStream_t s, cudaEvent_t* ev = nullptr);
// For every active system: cp = cr (start of a solve or restart, init = 1) or
// cp = cr + beta cp (a recurrence continued from the kept direction, init = 0); cr = 0.
template <typename T>
cudaError_t fused_prepare(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s,
                          int init = 1);

}  // namespace rpa
