// Row-tile form of the fused COCG direction + H-apply kernel (K_A of the fused iteration,
// Eq. 4 solved by COCG, Section 4), for grids whose x extent is at most 64 points.
//
// The column-tile kernel covers the xy plane with 32 x 8 tiles; on a 52-point or 40-point
// axis a quarter or more of its lanes then fall outside the grid.  Here a block owns TY
// complete x rows instead: its threads map linearly onto the nx x TY points of the tile, so
// every lane of every warp (up to the last partial warp) holds a grid point, and the
// R-point halo shrinks to R rows above and below plus the R-wide x padding of each row.
// Everything else follows the column-tile kernel: the block walks along z keeping the 2R+1
// values of each column in registers, the current xy plane (with halo) is double-buffered
// in shared memory and the next plane is prefetched while the current one is applied.  TY
// is chosen at run time by the autotuner among the heights row_candidates() lists.
#include <cuda_runtime.h>

#include <mutex>

#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kRowMaxHalo = 2;  // halo elements per thread
constexpr int kRowThreadsF32 = 768, kRowThreadsF64 = 512;

template <typename T>
constexpr int row_max_threads() {
  return sizeof(T) == 4 ? kRowThreadsF32 : kRowThreadsF64;
}

template <typename T, int R, bool FIRST>
__global__ void __launch_bounds__(row_max_threads<T>())
    k_dirmatvec_rows(CocgView<T> cv, FusedBufs<T> fb, int ty) {
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int EXN = nx + 2 * R;
  const int PLN = EXN * (ty + 2 * R);
  const int nthr = nx * ty;
  const int NHALO = PLN - nthr;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  cpx<T>* pl = reinterpret_cast<cpx<T>*>(dyn_smem);  // two planes with halo
  __shared__ T sh[32 * 2];
  const int ty0 = blockIdx.x * ty;
  const int z0 = blockIdx.z * fb.zchunk, z1 = min(z0 + fb.zchunk, nz);
  const int tid = threadIdx.x;
  const bool inblk = tid < nthr;
  const int lx = tid % nx, ly = tid / nx;
  const int gy = ty0 + ly;
  const bool valid = inblk && gy < ny;
  const long long sbase = (long long)s * cv.nd;
  const cpx<T>* __restrict__ r = cv.r + sbase;
  const cpx<T>* __restrict__ po = fb.p_in + sbase;
  cpx<T>* __restrict__ pn = fb.p_out + sbase;
  cpx<T>* __restrict__ w = cv.w + sbase;
  const T* __restrict__ vloc = cv.vloc;
  const double* sd = cv.sysd + (long long)s * kSysD;
  const cpx<T> be = mk<T>((T)sd[kBeta], (T)sd[kBeta + 1]);
  const int b = s / cv.ns, n = s - b * cv.ns;
  const cpx<T> sigma = mk<T>((T)cv.eps[n], (T)cv.omega[b]);
  // in-plane offsets of this thread's own point and of its halo elements (fixed along z)
  int own_xy = -1;
  if (inblk) {
    const int y = wrap_or_neg(gy, ny, st.bcy);
    own_xy = (y < 0) ? -1 : lx + nx * y;
  }
  // halo element hi -> its shared-memory slot and in-plane grid offset (-1: outside a
  // Dirichlet boundary).  Order: R full rows above, the 2R padding points of each tile row,
  // R full rows below.
  auto halo_pos = [&](int hi, int& slot, int& xy) {
    int ey, ex;
    if (hi < R * EXN) {
      ey = hi / EXN;
      ex = hi - ey * EXN;
    } else if (hi < R * EXN + ty * 2 * R) {
      const int t = hi - R * EXN;
      ey = R + t / (2 * R);
      const int c = t - (ey - R) * 2 * R;
      ex = (c < R) ? c : nx + c;
    } else {
      const int t = hi - R * EXN - ty * 2 * R;
      ey = R + ty + t / EXN;
      ex = t - (ey - R - ty) * EXN;
    }
    slot = ey * EXN + ex;
    const int x = wrap_or_neg(ex - R, nx, st.bcx), y = wrap_or_neg(ty0 - R + ey, ny, st.bcy);
    xy = (x < 0 || y < 0) ? -1 : x + nx * y;
  };
  // the first kRowMaxHalo halo elements of each thread are prefetched one plane ahead; the
  // rest (only on narrow grids, where the halo outgrows the tile) are loaded in place
  int halo_xy[kRowMaxHalo], halo_slot[kRowMaxHalo];
#pragma unroll
  for (int k = 0; k < kRowMaxHalo; ++k) {
    const int hi = tid + k * (int)blockDim.x;
    halo_slot[k] = -1;
    halo_xy[k] = -1;
    if (hi < NHALO) halo_pos(hi, halo_slot[k], halo_xy[k]);
  }
  const int own_slot = (ly + R) * EXN + (lx + R);
  auto zoff = [&](int z) -> int {
    const int zz = wrap_or_neg(z, nz, st.bcz);
    return zz < 0 ? -1 : zz * plane;
  };
  auto ld = [&](int q, cpx<T>& rv, cpx<T>& pv) {
    if (q < 0) {
      rv = mk<T>((T)0, (T)0);
      pv = rv;
    } else {
      rv = r[q];
      if (!FIRST) pv = po[q];
    }
  };
  auto comb = [&](const cpx<T>& rv, const cpx<T>& pv) -> cpx<T> {
    if (FIRST) return rv;
    return cadd(rv, cmul(be, pv));
  };
  cpx<T> zq[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    cpx<T> rv, pv;
    ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, rv, pv);
    zq[i] = comb(rv, pv);
  }
  cpx<T> nq_r, nq_p, h_r[kRowMaxHalo], h_p[kRowMaxHalo];
  auto prefetch = [&](int z) {
    const int zo = zoff(z + R);
    ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, nq_r, nq_p);
    const int zp = z * plane;
#pragma unroll
    for (int k = 0; k < kRowMaxHalo; ++k) ld(halo_xy[k] < 0 ? -1 : zp + halo_xy[k], h_r[k], h_p[k]);
  };
  if (z0 < z1) prefetch(z0);
  using A = dacc_t<T>;
  A acc_re = 0, acc_im = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    const int bo = ((z - z0) & 1) * PLN;
    zq[2 * R] = comb(nq_r, nq_p);
    if (inblk) pl[bo + own_slot] = zq[R];
#pragma unroll
    for (int k = 0; k < kRowMaxHalo; ++k)
      if (halo_slot[k] >= 0) pl[bo + halo_slot[k]] = comb(h_r[k], h_p[k]);
    for (int hi = tid + kRowMaxHalo * (int)blockDim.x; hi < NHALO; hi += blockDim.x) {
      int slot, xy;
      halo_pos(hi, slot, xy);
      cpx<T> rv, pv;
      ld(xy < 0 ? -1 : z * plane + xy, rv, pv);
      pl[bo + slot] = comb(rv, pv);
    }
    if (z + 1 < z1) prefetch(z + 1);
    __syncthreads();
    if (valid) {
      const int q = own_xy + z * plane;
      const cpx<T> c = zq[R];
      const cpx<T>* cs = pl + bo + own_slot;
      const T dg = c0 + vloc[q];
      cpx<T> a = mk<T>(dg * c.re - (sigma.re * c.re - sigma.im * c.im),
                       dg * c.im - (sigma.re * c.im + sigma.im * c.re));
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        a = caxpy_r(a, st.cx[m], cadd(cs[-m], cs[m]));
        a = caxpy_r(a, st.cy[m], cadd(cs[-m * EXN], cs[m * EXN]));
        a = caxpy_r(a, st.cz[m], cadd(zq[R - m], zq[R + m]));
      }
      w[q] = a;
      pn[q] = c;
      acc_re += (A)c.re * a.re - (A)c.im * a.im;
      acc_im += (A)c.re * a.im + (A)c.im * a.re;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) zq[i] = zq[i + 1];
  }
  A acc2[2] = {acc_re, acc_im};
  __shared__ A sha[32 * 2];
  block_sum_t<A, 2>(acc2, sha);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = (double)acc2[0];
    pp[1] = (double)acc2[1];
  }
}

template <typename T, int R>
void launch_r(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s) {
  const int ty = fb.row_ty;
  const dim3 grid(fb.ntiles_xy, fb.nact, fb.nzchunk);
  const int thr = ((cv.st.nx * ty + 31) / 32) * 32;
  const size_t pls = 2 * sizeof(cpx<T>) * (size_t)(cv.st.nx + 2 * R) * (ty + 2 * R);
  if (fb.first)
    k_dirmatvec_rows<T, R, true><<<grid, thr, pls, s>>>(cv, fb, ty);
  else
    k_dirmatvec_rows<T, R, false><<<grid, thr, pls, s>>>(cv, fb, ty);
}

constexpr int kRowSmemMax = 160 * 1024;

// opt-in dynamic shared memory of the row kernels, once per device and precision
template <typename T>
cudaError_t rows_attr() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
#define RPA_ROWS_ATTR(RR)                                                                      \
  if (e == cudaSuccess)                                                                        \
    e = cudaFuncSetAttribute(k_dirmatvec_rows<T, RR, true>,                                    \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kRowSmemMax);        \
  if (e == cudaSuccess)                                                                        \
    e = cudaFuncSetAttribute(k_dirmatvec_rows<T, RR, false>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kRowSmemMax);
  RPA_ROWS_ATTR(1) RPA_ROWS_ATTR(2) RPA_ROWS_ATTR(3) RPA_ROWS_ATTR(4)
  RPA_ROWS_ATTR(5) RPA_ROWS_ATTR(6) RPA_ROWS_ATTR(7) RPA_ROWS_ATTR(8)
#undef RPA_ROWS_ATTR
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

}  // namespace

template <typename T>
bool row_tile_fits(int nx, int ny, int R, int ty) {
  if (nx > 64 || R < 1 || R > 8 || ty < 1 || ty > ny) return false;
  const int thr = ((nx * ty + 31) / 32) * 32;
  if (thr > row_max_threads<T>()) return false;
  // two planes with halo
  const size_t pls = 2 * sizeof(cpx<T>) * (size_t)(nx + 2 * R) * (ty + 2 * R);
  return pls <= (size_t)kRowSmemMax;
}
template bool row_tile_fits<float>(int, int, int, int);
template bool row_tile_fits<double>(int, int, int, int);

template <typename T>
int row_candidates(int nx, int ny, int R, int ngroup, int* out, int maxn) {
  (void)ngroup;
  int cnt = 0;
  for (int ty = 2; ty <= ny && cnt < maxn; ++ty) {
    if (!row_tile_fits<T>(nx, ny, R, ty)) continue;
    const int thr = ((nx * ty + 31) / 32) * 32;
    // every halo element prefetched
    if ((nx + 2 * R) * (ty + 2 * R) - nx * ty > kRowMaxHalo * thr) continue;
    // heights that leave the last tile at least half full
    const int nt = (ny + ty - 1) / ty;
    if (2 * (nt * ty - ny) > ty) continue;
    // at least 3/4 of the threads of a block hold a grid point
    if (4 * nx * ty < 3 * thr) continue;
    out[cnt++] = ty;
  }
  return cnt;
}
template int row_candidates<float>(int, int, int, int, int*, int);
template int row_candidates<double>(int, int, int, int, int*, int);

template <typename T>
cudaError_t launch_dirmatvec_rows_prepare() {
  return rows_attr<T>();
}
template cudaError_t launch_dirmatvec_rows_prepare<float>();
template cudaError_t launch_dirmatvec_rows_prepare<double>();

template <typename T>
cudaError_t launch_dirmatvec_rows(const CocgView<T>& cv, const FusedBufs<T>& fb,
                                  cudaStream_t s) {
  cudaError_t e = rows_attr<T>();
  if (e != cudaSuccess) return e;
  switch (cv.st.R) {
    case 1: launch_r<T, 1>(cv, fb, s); break;
    case 2: launch_r<T, 2>(cv, fb, s); break;
    case 3: launch_r<T, 3>(cv, fb, s); break;
    case 4: launch_r<T, 4>(cv, fb, s); break;
    case 5: launch_r<T, 5>(cv, fb, s); break;
    case 6: launch_r<T, 6>(cv, fb, s); break;
    case 7: launch_r<T, 7>(cv, fb, s); break;
    default: launch_r<T, 8>(cv, fb, s); break;
  }
  return cudaGetLastError();
}
template cudaError_t launch_dirmatvec_rows<float>(const CocgView<float>&,
                                                  const FusedBufs<float>&, cudaStream_t);
template cudaError_t launch_dirmatvec_rows<double>(const CocgView<double>&,
                                                   const FusedBufs<double>&, cudaStream_t);

}  // namespace rpa
