// Fused COCG iteration for the batched Sternheimer systems (Eq. 4, Section 4).
//
// Per iteration and active system (unconjugated bilinear form a^T b):
//   K_A  p_k = r_k + beta_{k-1} p_{k-1};  w = (H - sigma) p_k;  partial mu = p_k^T w
//   S1   alpha = rho / mu
//   K_B  x += alpha p_k;  r -= alpha w;  partials ||r||^2, r^T r;  projector sums of r
//   S2   convergence test, beta = rho'/rho, projector coefficients of the next direction
// K_A is blocked in 2.5 dimensions: a block owns a 32 x 8 column tile of the grid and walks
// along z, keeping the 2R+1 values of its column in registers and the current xy plane
// (with an R-wide halo) in shared memory, so every input value is read from memory about
// once.  The direction vector is double-buffered (read p_{k-1}, write p_k) because
// neighbouring blocks read p_{k-1} in their halo.  The nonlocal term uses the projector
// coefficients of p_k, formed linearly from those of r_k and p_{k-1} by S2.
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "cocg_fused.cuh"

namespace rpa {

namespace {

__device__ __forceinline__ int wrap_or_neg(int j, int n, int bc) {
  if (bc == 0) {
    while (j < 0) j += n;
    while (j >= n) j -= n;
    return j;
  }
  return (j < 0 || j >= n) ? -1 : j;
}

template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[wid * NQ + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w)
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] += sh[w * NQ + q];
}

}  // namespace

constexpr int kFTX = 32, kFTY = 8;

// p_new at one grid point (or zero outside a Dirichlet boundary)
template <typename T>
__device__ __forceinline__ cpx<T> pnew_at(const cpx<T>* __restrict__ r, const cpx<T>* __restrict__ po,
                                          cpx<T> be, bool first, int gx, int gy, int gz,
                                          const Stencil<T>& st) {
  const int x = wrap_or_neg(gx, st.nx, st.bcx), y = wrap_or_neg(gy, st.ny, st.bcy),
            z = wrap_or_neg(gz, st.nz, st.bcz);
  if (x < 0 || y < 0 || z < 0) return mk<T>((T)0, (T)0);
  const long long q = x + (long long)st.nx * (y + (long long)st.ny * z);
  const cpx<T> rv = r[q];
  if (first) return rv;
  return cadd(rv, cmul(be, po[q]));
}

template <typename T, int R>
__global__ void __launch_bounds__(kFTX * kFTY) k_dirmatvec(CocgView<T> cv, FusedBufs<T> fb) {
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  __shared__ cpx<T> pl[kFTY + 2 * R][kFTX + 2 * R];
  __shared__ double sh[8 * 2];
  const Stencil<T>& st = cv.st;
  const int ntx = (st.nx + kFTX - 1) / kFTX;
  const int tile = blockIdx.x;
  const int tx0 = (tile % ntx) * kFTX, ty0 = (tile / ntx) * kFTY;
  const int zc = blockIdx.z;
  const int z0 = zc * fb.zchunk, z1 = min(z0 + fb.zchunk, st.nz);
  const int lx = threadIdx.x & (kFTX - 1), ly = threadIdx.x / kFTX;
  const int gx = tx0 + lx, gy = ty0 + ly;
  const bool valid = gx < st.nx && gy < st.ny;
  const long long nd = cv.nd;
  const cpx<T>* r = cv.r + (long long)s * nd;
  const cpx<T>* po = fb.p_in + (long long)s * nd;
  cpx<T>* pn = fb.p_out + (long long)s * nd;
  cpx<T>* w = cv.w + (long long)s * nd;
  const double* sd = cv.sysd + (long long)s * kSysD;
  const cpx<T> be = mk<T>((T)sd[kBeta], (T)sd[kBeta + 1]);
  const bool first = fb.first != 0;
  const int b = s / cv.ns, n = s - b * cv.ns;
  const cpx<T> sigma = mk<T>((T)cv.eps[n], (T)cv.omega[b]);
  const cpx<T>* cd = fb.cp + (long long)s * cv.nl.ngroup * kProjChunk;
  cpx<T> zq[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) zq[i] = pnew_at(r, po, be, first, gx, gy, z0 - R + i, st);
  double acc2[2] = {0.0, 0.0};
  const int ex_n = kFTX + 2 * R, ey_n = kFTY + 2 * R;
  for (int z = z0; z < z1; ++z) {
    zq[2 * R] = pnew_at(r, po, be, first, gx, gy, z + R, st);
    // current plane into shared memory: own value, then the halo ring
    pl[ly + R][lx + R] = zq[R];
    for (int e = threadIdx.x; e < ex_n * ey_n; e += blockDim.x) {
      const int ey = e / ex_n, ex = e - ey * ex_n;
      if (ey >= R && ey < R + kFTY && ex >= R && ex < R + kFTX) continue;
      pl[ey][ex] = pnew_at(r, po, be, first, tx0 - R + ex, ty0 - R + ey, z, st);
    }
    __syncthreads();
    if (valid) {
      const long long q = gx + (long long)st.nx * (gy + (long long)st.ny * z);
      const cpx<T> c = zq[R];
      const T dg = st.c0 + cv.vloc[q];
      cpx<T> a = mk<T>(dg * c.re - (sigma.re * c.re - sigma.im * c.im),
                       dg * c.im - (sigma.re * c.im + sigma.im * c.re));
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        a = caxpy_r(a, st.cx[m], cadd(pl[ly + R][lx + R - m], pl[ly + R][lx + R + m]));
        a = caxpy_r(a, st.cy[m], cadd(pl[ly + R - m][lx + R], pl[ly + R + m][lx + R]));
        a = caxpy_r(a, st.cz[m], cadd(zq[R - m], zq[R + m]));
      }
      if (cv.nl.ngroup > 0) {
        const int e0 = cv.nl.p_off[q], e1 = cv.nl.p_off[q + 1];
        for (int e = e0; e < e1; ++e) {
          const int g = cv.nl.p_grp[e];
          const T* ch = cv.nl.p_chi + (long long)e * kProjChunk;
          const cpx<T>* cg = cd + (long long)g * kProjChunk;
#pragma unroll
          for (int l = 0; l < kProjChunk; ++l) a = caxpy_r(a, ch[l], cg[l]);
        }
      }
      w[q] = a;
      pn[q] = c;
      acc2[0] += (double)c.re * a.re - (double)c.im * a.im;
      acc2[1] += (double)c.re * a.im + (double)c.im * a.re;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) zq[i] = zq[i + 1];
  }
  block_sum<2>(acc2, sh);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = acc2[0];
    pp[1] = acc2[1];
  }
}

// x += alpha p, r -= alpha w; partials ||r||^2 (slot 0) and r^T r (slots 2, 3).  The
// updated r of the tile is kept in shared memory; then each warp takes whole projector
// groups touching the tile (their entries are sorted by grid index, so a group's entries in
// this tile are one contiguous range), reduces coef * chi * r over the range with shuffles
// and adds the tile's contribution to cr[s][g][l] with one atomic per value.
template <typename T>
__global__ void __launch_bounds__(256) k_update_dots(CocgView<T> cv, FusedBufs<T> fb) {
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  __shared__ double sh[8 * 3];
  __shared__ cpx<T> sr[kTile];
  const long long nd = cv.nd;
  const double* sd = cv.sysd + (long long)s * kSysD;
  const cpx<T> al = mk<T>((T)sd[kAlpha], (T)sd[kAlpha + 1]);
  const bool nl = cv.nl.ngroup > 0;
  double acc[3] = {0.0, 0.0, 0.0};
  const long long t0 = (long long)blockIdx.x * kTile;
  const long long t1 = min(t0 + kTile, nd);
  for (long long p = t0 + threadIdx.x; p < t1; p += blockDim.x) {
    const long long q = (long long)s * nd + p;
    const cpx<T> pv = fb.p_out[q], wv = cv.w[q];
    cv.x[q] = cadd(cv.x[q], cmul(al, pv));
    const cpx<T> rv = csub(cv.r[q], cmul(al, wv));
    cv.r[q] = rv;
    if (nl) sr[p - t0] = rv;
    acc[0] += (double)rv.re * rv.re + (double)rv.im * rv.im;
    acc[1] += (double)rv.re * rv.re - (double)rv.im * rv.im;
    acc[2] += 2.0 * (double)rv.re * rv.im;
  }
  if (nl) {
    __syncthreads();
    cpx<T>* cr = fb.cr + (long long)s * cv.nl.ngroup * kProjChunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q0 = fb.tile_roff[blockIdx.x], q1 = fb.tile_roff[blockIdx.x + 1];
    for (int q = q0 + warp; q < q1; q += (int)(blockDim.x >> 5)) {
      const int g = fb.tile_ranges[3 * q], e0 = fb.tile_ranges[3 * q + 1],
                e1 = fb.tile_ranges[3 * q + 2];
      T a[2 * kProjChunk];
#pragma unroll
      for (int i = 0; i < 2 * kProjChunk; ++i) a[i] = (T)0;
      for (int e = e0 + lane; e < e1; e += 32) {
        const cpx<T> rv = sr[cv.nl.g_idx[e] - t0];
        const T* ch = cv.nl.g_chi + (long long)e * kProjChunk;
#pragma unroll
        for (int l = 0; l < kProjChunk; ++l) {
          a[2 * l] += ch[l] * rv.re;
          a[2 * l + 1] += ch[l] * rv.im;
        }
      }
#pragma unroll
      for (int i = 0; i < 2 * kProjChunk; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_down_sync(0xffffffffu, a[i], o);
      if (lane < kProjChunk) {
        T re = a[0], im = a[1];
#pragma unroll
        for (int l = 1; l < kProjChunk; ++l)
          if (lane == l) {
            re = a[2 * l];
            im = a[2 * l + 1];
          }
        const T cf = cv.nl.coef[g * kProjChunk + lane];
        atomicAdd(&cr[g * kProjChunk + lane].re, cf * re);
        atomicAdd(&cr[g * kProjChunk + lane].im, cf * im);
      }
    }
  }
  block_sum<3>(acc, sh);
  if (threadIdx.x == 0) {
    double* pp = cv.part + ((long long)s * cv.tiles + blockIdx.x) * 4;
    pp[0] = acc[0];
    pp[2] = acc[1];
    pp[3] = acc[2];
  }
}

// S2 with the projector bookkeeping: after the scalar step (kind 2), every still-active
// system forms cp = cr + beta cp and clears cr.  One warp per system.
template <typename T>
__global__ void k_proj_next(int nsys, int ngroup, const double* __restrict__ sysd,
                            const int* __restrict__ sysi, int init, cpx<T>* __restrict__ cp,
                            cpx<T>* __restrict__ cr, const int* __restrict__ list) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nsys) return;
  const int s = list ? list[i] : i;
  if (sysi[(long long)s * kSysI + kStatus] != kActive) return;
  const double* sd = sysd + (long long)s * kSysD;
  const cpx<T> be = init ? mk<T>((T)0, (T)0) : mk<T>((T)sd[kBeta], (T)sd[kBeta + 1]);
  cpx<T>* p = cp + (long long)s * ngroup * kProjChunk;
  cpx<T>* q = cr + (long long)s * ngroup * kProjChunk;
  for (int i = lane; i < ngroup * kProjChunk; i += 32) {
    p[i] = init ? q[i] : cadd(q[i], cmul(be, p[i]));
    q[i] = mk<T>((T)0, (T)0);
  }
}

// -------------------------------------------------------------------------------------------
template <typename T, int R>
static void launch_dirmatvec(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s) {
  dim3 grid(fb.ntiles_xy, fb.nact, fb.nzchunk);
  k_dirmatvec<T, R><<<grid, kFTX * kFTY, 0, s>>>(cv, fb);
}

template <typename T>
cudaError_t fused_iteration(const CocgView<T>& cv, const FusedBufs<T>& fb, double tol, int maxit,
                            cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  if (ev) cudaEventRecord(ev[1], s);
  switch (cv.st.R) {
    case 1: launch_dirmatvec<T, 1>(cv, fb, s); break;
    case 2: launch_dirmatvec<T, 2>(cv, fb, s); break;
    case 3: launch_dirmatvec<T, 3>(cv, fb, s); break;
    case 4: launch_dirmatvec<T, 4>(cv, fb, s); break;
    case 5: launch_dirmatvec<T, 5>(cv, fb, s); break;
    case 6: launch_dirmatvec<T, 6>(cv, fb, s); break;
    case 7: launch_dirmatvec<T, 7>(cv, fb, s); break;
    default: launch_dirmatvec<T, 8>(cv, fb, s); break;
  }
  if (ev) cudaEventRecord(ev[2], s);
  cudaError_t e = cocg_scalars(fb.nact, fb.ntiles_xy * fb.nzchunk, cv.part, cv.sysd, cv.sysi, 1,
                               1 << kActive, tol, 0.0, maxit, 0, s, cv.tiles, cv.list);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  dim3 g2(fb.tiles1d, fb.nact);
  k_update_dots<T><<<g2, 256, 0, s>>>(cv, fb);
  if (ev) cudaEventRecord(ev[4], s);
  e = cocg_scalars(fb.nact, fb.tiles1d, cv.part, cv.sysd, cv.sysi, 2, 1 << kActive, tol, 0.0,
                   maxit, 0, s, cv.tiles, cv.list);
  if (e != cudaSuccess) return e;
  if (cv.nl.ngroup > 0) {
    k_proj_next<T><<<(fb.nact + 3) / 4, 128, 0, s>>>(fb.nact, cv.nl.ngroup, cv.sysd, cv.sysi, 0,
                                                     fb.cp, fb.cr, cv.list);
    note_launch();
  }
  if (ev) cudaEventRecord(ev[5], s);
  if (ev) cudaEventRecord(ev[6], s);
  note_launch(2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fused_prepare(const CocgView<T>& cv, const FusedBufs<T>& fb, cudaStream_t s) {
  if (cv.nl.ngroup == 0) return cudaSuccess;
  k_proj_next<T><<<(cv.nsys + 3) / 4, 128, 0, s>>>(cv.nsys, cv.nl.ngroup, cv.sysd, cv.sysi, 1,
                                                   fb.cp, fb.cr, nullptr);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t fused_iteration<double>(const CocgView<double>&, const FusedBufs<double>&,
                                             double, int, cudaStream_t, cudaEvent_t*);
template cudaError_t fused_iteration<float>(const CocgView<float>&, const FusedBufs<float>&,
                                            double, int, cudaStream_t, cudaEvent_t*);
template cudaError_t fused_prepare<double>(const CocgView<double>&, const FusedBufs<double>&,
                                           cudaStream_t);
template cudaError_t fused_prepare<float>(const CocgView<float>&, const FusedBufs<float>&,
                                          cudaStream_t);

}  // namespace rpa
