// True residual r = b - (H - sigma) x of the Sternheimer systems (Eq. 4) with
// b_n = -psi_n (.) u, in the 2.5-D blocked form of the fused COCG kernels: a block owns a
// 32 x 8 column tile, walks z with the 2R+1 values of its column in registers and the current
// xy plane (with an R-wide halo) in shared memory, next plane prefetched.  Used for the
// initial residual of every solve, the true-residual recheck of the FP64 form and the FP64
// residual of each refinement round of the mixed form (T = double, low-precision copies of r
// in TL = float for the next FP32 round).  Partial sums per tile: ||r||^2, ||b||^2 and
// r^T r (re, im); partial slots beyond this launch's tiles are zeroed so that a per-system
// sum over the full partial stride sees only this launch.
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kRTX = 32, kRTY = 8;

template <typename T, typename TL, int R, bool SMEM_CD>
__global__ void __launch_bounds__(kRTX * kRTY, sizeof(T) == 4 ? 3 : 2)
    k_resid_fused(CocgView<T> cv, const cpx<T>* __restrict__ x, cpx<T>* __restrict__ r,
                  cpx<T>* __restrict__ pdir, int mask, cpx<TL>* __restrict__ r_lo,
                  cpx<TL>* __restrict__ p_lo, cpx<TL>* __restrict__ x_lo, int zchunk) {
  const int s = blockIdx.y;
  const int st_s = cv.sysi[(long long)s * kSysI + kStatus];
  if (!((mask >> st_s) & 1)) return;
  constexpr int EXN = kRTX + 2 * R, EYN = kRTY + 2 * R;
  constexpr int PLN = EXN * EYN;
  constexpr int NHALO = PLN - kRTX * kRTY;
  constexpr int HPT = (NHALO + kRTX * kRTY - 1) / (kRTX * kRTY);
  __shared__ cpx<T> pl[2 * PLN];
  __shared__ T sh[8 * 4];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int ntx = (nx + kRTX - 1) / kRTX;
  const int tx0 = (blockIdx.x % ntx) * kRTX, ty0 = (blockIdx.x / ntx) * kRTY;
  const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, nz);
  const int lx = threadIdx.x & (kRTX - 1), ly = threadIdx.x / kRTX;
  const int gx = tx0 + lx, gy = ty0 + ly;
  const bool valid = gx < nx && gy < ny;
  const long long sbase = (long long)s * cv.nd;
  const cpx<T>* __restrict__ xs = x + sbase;
  const T* __restrict__ vloc = cv.vloc;
  const int b = s / cv.ns, n = s - b * cv.ns;
  const cpx<T> sigma = mk<T>((T)cv.eps[n], (T)cv.omega[b]);
  const T* __restrict__ psin = cv.psi + (long long)n * cv.nd;
  const T* __restrict__ ub = cv.u + (long long)b * cv.nd;
  const int ncd = cv.nl.ngroup * kProjChunk;
  const cpx<T>* cd = cv.cdot + (long long)s * ncd;
  if (SMEM_CD) {
    cpx<T>* scd = reinterpret_cast<cpx<T>*>(dyn_smem);
    for (int i = threadIdx.x; i < ncd; i += blockDim.x) scd[i] = cd[i];
    cd = scd;  // read after the first barrier of the z loop
  }
  // partial slots past this launch's tiles: zeroed by the first block of the system
  if (blockIdx.x == 0 && blockIdx.z == 0) {
    const int used = gridDim.x * gridDim.z;
    double* pp = cv.part + (long long)s * cv.tiles * 4;
    for (int i = used * 4 + threadIdx.x; i < cv.tiles * 4; i += blockDim.x) pp[i] = 0.0;
  }
  int own_xy;
  {
    const int xx = wrap_or_neg(gx, nx, st.bcx), yy = wrap_or_neg(gy, ny, st.bcy);
    own_xy = (xx < 0 || yy < 0) ? -1 : xx + nx * yy;
  }
  int halo_xy[HPT], halo_slot[HPT];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int hi = threadIdx.x + k * kRTX * kRTY;
    halo_slot[k] = -1;
    halo_xy[k] = -1;
    if (hi < NHALO) {
      // R rows above, the 2R padding points of each tile row, R rows below
      int ey, ex;
      if (hi < R * EXN) {
        ey = hi / EXN;
        ex = hi - ey * EXN;
      } else if (hi < R * EXN + kRTY * 2 * R) {
        const int t = hi - R * EXN;
        ey = R + t / (2 * R);
        const int c = t - (ey - R) * 2 * R;
        ex = (c < R) ? c : kRTX + c;
      } else {
        const int t = hi - R * EXN - kRTY * 2 * R;
        ey = R + kRTY + t / EXN;
        ex = t - (ey - R - kRTY) * EXN;
      }
      halo_slot[k] = ey * EXN + ex;
      const int xx = wrap_or_neg(tx0 - R + ex, nx, st.bcx),
                yy = wrap_or_neg(ty0 - R + ey, ny, st.bcy);
      halo_xy[k] = (xx < 0 || yy < 0) ? -1 : xx + nx * yy;
    }
  }
  const int own_slot = (ly + R) * EXN + (lx + R);
  auto zoff = [&](int z) -> int {
    const int zz = wrap_or_neg(z, nz, st.bcz);
    return zz < 0 ? -1 : zz * plane;
  };
  auto ld = [&](int q) -> cpx<T> { return q < 0 ? mk<T>((T)0, (T)0) : xs[q]; };
  cpx<T> zq[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    zq[i] = ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy);
  }
  cpx<T> nq, hv[HPT];
  const bool has_nl = cv.nl.ngroup > 0;
  const int* __restrict__ p_off = cv.nl.p_off;
  const int* __restrict__ p_grp = cv.nl.p_grp;
  const T* __restrict__ p_chi = cv.nl.p_chi;
  int ne0 = 0, ne1 = 0;
  auto prefetch = [&](int z) {
    const int zo = zoff(z + R);
    nq = ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy);
    const int zp = z * plane;
#pragma unroll
    for (int k = 0; k < HPT; ++k) hv[k] = ld(halo_xy[k] < 0 ? -1 : zp + halo_xy[k]);
    if (has_nl && valid) {
      const int q = own_xy + zp;
      ne0 = p_off[q];
      ne1 = p_off[q + 1];
    }
  };
  if (z0 < z1) prefetch(z0);
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    const int bo = ((z - z0) & 1) * PLN;
    zq[2 * R] = nq;
    pl[bo + own_slot] = zq[R];
#pragma unroll
    for (int k = 0; k < HPT; ++k)
      if (halo_slot[k] >= 0) pl[bo + halo_slot[k]] = hv[k];
    const int e0 = ne0, e1 = ne1;
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
      for (int e = e0; e < e1; ++e) {
        const int g = p_grp[e];
        T ch[kProjChunk];
        load_chi4(p_chi + kProjChunk * e, ch);
        const cpx<T>* cg = cd + kProjChunk * g;
#pragma unroll
        for (int l = 0; l < kProjChunk; ++l) a = caxpy_r(a, ch[l], cg[l]);
      }
      const cpx<T> bv = mk<T>(-psin[q] * ub[q], (T)0);
      const cpx<T> rv = csub(bv, a);
      r[sbase + q] = rv;
      if (pdir) pdir[sbase + q] = rv;
      if (r_lo) {
        const cpx<TL> rl = mk<TL>((TL)rv.re, (TL)rv.im);
        r_lo[sbase + q] = rl;
        p_lo[sbase + q] = rl;
        x_lo[sbase + q] = mk<TL>((TL)0, (TL)0);
      }
      a0 += rv.re * rv.re + rv.im * rv.im;
      a1 += bv.re * bv.re;
      a2 += rv.re * rv.re - rv.im * rv.im;
      a3 += (T)2 * rv.re * rv.im;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) zq[i] = zq[i + 1];
  }
  T acc[4] = {a0, a1, a2, a3};
  block_sum_t<T, 4>(acc, sh);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) pp[q] = (double)acc[q];
  }
}

template <typename T, typename TL, int R>
void launch_r(const CocgView<T>& cv, const cpx<T>* x, cpx<T>* r, cpx<T>* pdir, int mask,
              cpx<TL>* r_lo, cpx<TL>* p_lo, cpx<TL>* x_lo, cudaStream_t s) {
  constexpr size_t kPlanes = 2 * sizeof(cpx<T>) * (kRTX + 2 * R) * (kRTY + 2 * R);
  size_t cdb = sizeof(cpx<T>) * cv.nl.ngroup * kProjChunk;
  if (cdb + kPlanes + 1024 > 48 * 1024) cdb = 0;
  const int nx = cv.st.nx, ny = cv.st.ny, nz = cv.st.nz;
  const int zchunk = nz <= 64 ? nz : 32;
  const dim3 grid(((nx + kRTX - 1) / kRTX) * ((ny + kRTY - 1) / kRTY), cv.nsys,
                  (nz + zchunk - 1) / zchunk);
  if (cdb)
    k_resid_fused<T, TL, R, true><<<grid, kRTX * kRTY, cdb, s>>>(cv, x, r, pdir, mask, r_lo,
                                                                   p_lo, x_lo, zchunk);
  else
    k_resid_fused<T, TL, R, false><<<grid, kRTX * kRTY, 0, s>>>(cv, x, r, pdir, mask, r_lo,
                                                                  p_lo, x_lo, zchunk);
}

}  // namespace

template <typename T, typename TL>
cudaError_t cocg_resid(const CocgView<T>& cv, const cpx<T>* x, cpx<T>* r, cpx<T>* pdir, int mask,
                       cpx<TL>* r_lo, cpx<TL>* p_lo, cpx<TL>* x_lo, cudaStream_t s) {
  const int nx = cv.st.nx, ny = cv.st.ny, nz = cv.st.nz;
  const int zchunk = nz <= 64 ? nz : 32;
  const long long used = (long long)((nx + kRTX - 1) / kRTX) * ((ny + kRTY - 1) / kRTY) *
                         ((nz + zchunk - 1) / zchunk);
  if (used > cv.tiles) return cudaErrorInvalidValue;  // partial buffer too small
  switch (cv.st.R) {
    case 1: launch_r<T, TL, 1>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 2: launch_r<T, TL, 2>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 3: launch_r<T, TL, 3>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 4: launch_r<T, TL, 4>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 5: launch_r<T, TL, 5>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 6: launch_r<T, TL, 6>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    case 7: launch_r<T, TL, 7>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
    default: launch_r<T, TL, 8>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, s); break;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t cocg_resid<double, double>(const CocgView<double>&, const cpx<double>*,
                                                cpx<double>*, cpx<double>*, int, cpx<double>*,
                                                cpx<double>*, cpx<double>*, cudaStream_t);
template cudaError_t cocg_resid<double, float>(const CocgView<double>&, const cpx<double>*,
                                               cpx<double>*, cpx<double>*, int, cpx<float>*,
                                               cpx<float>*, cpx<float>*, cudaStream_t);
template cudaError_t cocg_resid<float, float>(const CocgView<float>&, const cpx<float>*,
                                              cpx<float>*, cpx<float>*, int, cpx<float>*,
                                              cpx<float>*, cpx<float>*, cudaStream_t);

}  // namespace rpa
