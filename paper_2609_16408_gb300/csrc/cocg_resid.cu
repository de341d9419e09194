// True residual r = b - (H - sigma) x of the Sternheimer systems (Eq. 4) with
// b_n = -psi_n (.) u, in the 2.5-D blocked form of the fused COCG kernels: a block owns a
// 32 x 8 column tile, walks z with the 2R+1 values of its column in registers and the current
// xy plane (with an R-wide halo) in shared memory, next plane prefetched.  Used for the
// initial residual of every solve, the true-residual recheck of the FP64 form and the FP64
// residual of each refinement round of the mixed form (T = double, low-precision copies of r
// in TL = float for the next FP32 round).  Partial sums per tile: ||r||^2, ||b||^2 and
// r^T r (re, im); partial slots beyond this launch's tiles are zeroed so that a per-system
// sum over the full partial stride sees only this launch.
//
// With use_df (FP64 inputs; chosen by the caller when the solve tolerance leaves room for it)
// the 6R-neighbour part of the stencil, which dominates the arithmetic, runs in double-float
// arithmetic on the FP32 units (each value an unevaluated sum hi + lo of two floats; Dekker's
// exact product through FMA and Knuth's two-sum, about 48 significant bits, i.e. ~32x the
// FP64 rounding error) because FP64 runs at 1/58 of the FP32 rate on this GPU.  The diagonal,
// the projector terms, b and the sums stay in FP64.
#include <cuda_runtime.h>

#include <type_traits>

#include "cocg.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kRTX = 32, kRTY = 8;

// the stencil coefficients as double-float pairs (kernel parameters)
struct DfCoef {
  float hx[kMaxRadius + 1], lx[kMaxRadius + 1], hy[kMaxRadius + 1], ly[kMaxRadius + 1],
      hz[kMaxRadius + 1], lz[kMaxRadius + 1];
  float c0h, c0l;
};

// XDF (T = double, TL = float: the mixed form's refinement): x holds double-float pairs.
// DF (with XDF): the whole residual in double-float arithmetic on the FP32 units; without
// DF the loaded pairs are summed into FP64 and the FP64 arithmetic follows.
template <typename T, typename TL, int R, bool SMEM_CD, bool DF>
__global__ void __launch_bounds__(kRTX * kRTY, sizeof(T) == 4 ? 3 : 2)
    k_resid_fused(CocgView<T> cv, const cpx<T>* __restrict__ x, cpx<T>* __restrict__ r,
                  cpx<T>* __restrict__ pdir, int mask, cpx<TL>* __restrict__ r_lo,
                  cpx<TL>* __restrict__ p_lo, cpx<TL>* __restrict__ x_lo, int zchunk,
                  DfCoef dc, const cpx<TL>* __restrict__ p_keep, DfAux aux) {
  constexpr bool XDF = sizeof(T) == 8 && std::is_same<TL, float>::value;
  static_assert(!DF || XDF, "the double-float path is the mixed form's refinement");
  using V = typename std::conditional<DF, cdf, cpx<T>>::type;  // stored neighbour values
  using AT = typename std::conditional<DF, float, T>::type;    // partial sums
  const int s = blockIdx.y;
  const int st_s = cv.sysi[(long long)s * kSysI + kStatus];
  if (!((mask >> st_s) & 1)) return;
  // direction of the low-precision recurrence: 0 restart (p_lo = r_lo), 1 keep p_lo,
  // 2 copy the kept direction from p_keep (see cocg_resid)
  int pmode = 0;
  if (p_keep) {
    const int ran = cv.sysi[(long long)s * kSysI + kIters] - cv.sysi[(long long)s * kSysI + kIterBase];
    pmode = ran <= 0 ? 0 : ((ran & 1) ? 2 : 1);
  }
  constexpr int EXN = kRTX + 2 * R, EYN = kRTY + 2 * R;
  constexpr int PLN = EXN * EYN;
  constexpr int NHALO = PLN - kRTX * kRTY;
  constexpr int HPT = (NHALO + kRTX * kRTY - 1) / (kRTX * kRTY);
  __shared__ V pl[2 * PLN];
  __shared__ AT sh[8 * 4];
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
  const float4* __restrict__ xd = reinterpret_cast<const float4*>(x) + sbase;  // XDF
  const T* __restrict__ vloc = cv.vloc;
  const int b = s / cv.ns, n = s - b * cv.ns;
  const cpx<T> sigma = mk<T>((T)cv.eps[n], (T)cv.omega[b]);
  const T* __restrict__ psin = cv.psi + (long long)n * cv.nd;
  const T* __restrict__ ub = cv.u + (long long)b * cv.nd;
  const int ncd = cv.nl.ngroup * kProjChunk;
  const cpx<T>* cd = cv.cdot + (long long)s * ncd;
  const cdf* cdd = nullptr;  // DF: the coefficients as double-float pairs in shared memory
  if (SMEM_CD) {
    if constexpr (DF) {
      cdf* scd = reinterpret_cast<cdf*>(dyn_smem);
      for (int i = threadIdx.x; i < ncd; i += blockDim.x) scd[i] = cdf_of(cd[i]);
      cdd = scd;
    } else {
      cpx<T>* scd = reinterpret_cast<cpx<T>*>(dyn_smem);
      for (int i = threadIdx.x; i < ncd; i += blockDim.x) scd[i] = cd[i];
      cd = scd;  // read after the first barrier of the z loop
    }
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
  auto ld = [&](int q) -> V {
    if constexpr (DF) {
      return q < 0 ? cdf{df{0.f, 0.f}, df{0.f, 0.f}} : cdf_ld(xd[q]);
    } else if constexpr (XDF) {
      if (q < 0) return mk<T>((T)0, (T)0);
      const cdf v = cdf_ld(xd[q]);
      return mk<T>(df_val(v.re), df_val(v.im));
    } else {
      return q < 0 ? mk<T>((T)0, (T)0) : xs[q];
    }
  };
  V zq[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    zq[i] = ld((zo < 0 || own_xy < 0) ? -1 : zo + own_xy);
  }
  V nq, hv[HPT];
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
  AT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const T c0 = st.c0;
  // DF: sigma = eps_n + i omega_b as double-float pairs
  const df smr = df_of(-(double)cv.eps[n]), smi = df_of((double)cv.omega[b]);
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
      const V* cs = pl + bo + own_slot;
      if constexpr (DF) {
        // (H - sigma) x at q: neighbours, diagonal (c0 + V - sigma), projector terms and
        // b = -psi_n u, every product and sum in double-float arithmetic
        const cdf c = zq[R];
        df sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
        for (int m = 1; m <= R; ++m) {
          const df kx{dc.hx[m], dc.lx[m]}, ky{dc.hy[m], dc.ly[m]}, kz{dc.hz[m], dc.lz[m]};
          sr = df_fma(sr, kx, df_add(cs[-m].re, cs[m].re));
          si = df_fma(si, kx, df_add(cs[-m].im, cs[m].im));
          sr = df_fma(sr, ky, df_add(cs[-m * EXN].re, cs[m * EXN].re));
          si = df_fma(si, ky, df_add(cs[-m * EXN].im, cs[m * EXN].im));
          sr = df_fma(sr, kz, df_add(zq[R - m].re, zq[R + m].re));
          si = df_fma(si, kz, df_add(zq[R - m].im, zq[R + m].im));
        }
        const float2 vq = aux.vloc[q];
        const df dd = df_add(df_add(df{dc.c0h, dc.c0l}, df{vq.x, vq.y}), smr);  // c0 + V - Re sigma
        df are = df_add(df_fma(df_mul(dd, c.re), smi, c.im), sr);
        df aim = df_add(df_fma(df_mul(dd, c.im), df_neg(smi), c.re), si);
        for (int e = e0; e < e1; ++e) {
          const int g = p_grp[e];
          const cdf* cg = cdd ? cdd + kProjChunk * g : nullptr;
#pragma unroll
          for (int l = 0; l < kProjChunk; ++l) {
            const df ch{aux.nl.p_chi[kProjChunk * e + l], aux.p_chi_lo[kProjChunk * e + l]};
            const cdf cl = cg ? cg[l] : cdf_of(cd[kProjChunk * g + l]);
            are = df_fma(are, ch, cl.re);
            aim = df_fma(aim, ch, cl.im);
          }
        }
        const float2 pq = aux.psi[(long long)n * cv.nd + q], uq = aux.u[(long long)b * cv.nd + q];
        const df bre = df_neg(df_mul(df{pq.x, pq.y}, df{uq.x, uq.y}));
        const df rre = df_add(bre, df_neg(are)), rim = df_neg(aim);
        const float rr = __fadd_rn(rre.hi, rre.lo), ri = __fadd_rn(rim.hi, rim.lo);
        if (r) r[sbase + q] = mk<T>((T)df_val(rre), (T)df_val(rim));
        if (r_lo) {
          const cpx<TL> rl = mk<TL>((TL)rr, (TL)ri);
          r_lo[sbase + q] = rl;
          if (pmode == 0)
            p_lo[sbase + q] = rl;
          else if (pmode == 2)
            p_lo[sbase + q] = p_keep[sbase + q];
          x_lo[sbase + q] = mk<TL>((TL)0, (TL)0);
        }
        const float bv = __fadd_rn(bre.hi, bre.lo);
        a0 += rr * rr + ri * ri;
        a1 += bv * bv;
        a2 += rr * rr - ri * ri;
        a3 += 2.f * rr * ri;
      } else {
      const T dg = c0 + vloc[q];
      cpx<T> c, a;
      c = zq[R];
      a = mk<T>(dg * c.re - (sigma.re * c.re - sigma.im * c.im),
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
      if (r) r[sbase + q] = rv;
      if (pdir) pdir[sbase + q] = rv;
      if (r_lo) {
        const cpx<TL> rl = mk<TL>((TL)rv.re, (TL)rv.im);
        r_lo[sbase + q] = rl;
        if (pmode == 0)
          p_lo[sbase + q] = rl;
        else if (pmode == 2)
          p_lo[sbase + q] = p_keep[sbase + q];
        x_lo[sbase + q] = mk<TL>((TL)0, (TL)0);
      }
      a0 += rv.re * rv.re + rv.im * rv.im;
      a1 += bv.re * bv.re;
      a2 += rv.re * rv.re - rv.im * rv.im;
      a3 += (T)2 * rv.re * rv.im;
      }
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) zq[i] = zq[i + 1];
  }
  AT acc[4] = {a0, a1, a2, a3};
  block_sum_t<AT, 4>(acc, sh);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) pp[q] = (double)acc[q];
  }
}

template <typename T, typename TL, int R>
void launch_r(const CocgView<T>& cv, const cpx<T>* x, cpx<T>* r, cpx<T>* pdir, int mask,
              cpx<TL>* r_lo, cpx<TL>* p_lo, cpx<TL>* x_lo, bool use_df,
              const cpx<TL>* p_keep, const DfAux& aux, cudaStream_t s) {
  constexpr size_t kPlanes = 2 * sizeof(cpx<T>) * (kRTX + 2 * R) * (kRTY + 2 * R);
  size_t cdb = sizeof(cpx<T>) * cv.nl.ngroup * kProjChunk;
  if (cdb + kPlanes + 1024 > 48 * 1024) cdb = 0;
  const int nx = cv.st.nx, ny = cv.st.ny, nz = cv.st.nz;
  const int zchunk = nz <= 64 ? nz : 32;
  const dim3 grid(((nx + kRTX - 1) / kRTX) * ((ny + kRTY - 1) / kRTY), cv.nsys,
                  (nz + zchunk - 1) / zchunk);
  DfCoef dc{};
  if (use_df && sizeof(T) == 8) {  // hi + lo splits of the neighbour coefficients
    for (int m = 0; m <= R; ++m) {
      const double v[3] = {(double)cv.st.cx[m], (double)cv.st.cy[m], (double)cv.st.cz[m]};
      float* hi[3] = {dc.hx, dc.hy, dc.hz};
      float* lo[3] = {dc.lx, dc.ly, dc.lz};
      for (int a = 0; a < 3; ++a) {
        hi[a][m] = (float)v[a];
        lo[a][m] = (float)(v[a] - (double)hi[a][m]);
      }
    }
    dc.c0h = (float)(double)cv.st.c0;
    dc.c0l = (float)((double)cv.st.c0 - (double)dc.c0h);
  }
  if constexpr (sizeof(T) == 8 && std::is_same<TL, float>::value) {
    if (use_df) {
      if (cdb)
        k_resid_fused<T, TL, R, true, true><<<grid, kRTX * kRTY, cdb, s>>>(
            cv, x, r, pdir, mask, r_lo, p_lo, x_lo, zchunk, dc, p_keep, aux);
      else
        k_resid_fused<T, TL, R, false, true><<<grid, kRTX * kRTY, 0, s>>>(
            cv, x, r, pdir, mask, r_lo, p_lo, x_lo, zchunk, dc, p_keep, aux);
      return;
    }
  }
  if (cdb)
    k_resid_fused<T, TL, R, true, false><<<grid, kRTX * kRTY, cdb, s>>>(
        cv, x, r, pdir, mask, r_lo, p_lo, x_lo, zchunk, dc, p_keep, aux);
  else
    k_resid_fused<T, TL, R, false, false><<<grid, kRTX * kRTY, 0, s>>>(
        cv, x, r, pdir, mask, r_lo, p_lo, x_lo, zchunk, dc, p_keep, aux);
}

}  // namespace

template <typename T, typename TL>
cudaError_t cocg_resid(const CocgView<T>& cv, const cpx<T>* x, cpx<T>* r, cpx<T>* pdir, int mask,
                       cpx<TL>* r_lo, cpx<TL>* p_lo, cpx<TL>* x_lo, cudaStream_t s,
                       bool use_df, const cpx<TL>* p_keep, const DfAux* aux) {
  if (p_keep && !r_lo) return cudaErrorInvalidValue;
  constexpr bool kXdf = sizeof(T) == 8 && std::is_same<TL, float>::value;
  if (use_df && (!kXdf || !aux)) return cudaErrorInvalidValue;
  if (!kXdf && !r) return cudaErrorInvalidValue;
  const DfAux noaux{};
  const DfAux& ax = aux ? *aux : noaux;
  const int nx = cv.st.nx, ny = cv.st.ny, nz = cv.st.nz;
  const int zchunk = nz <= 64 ? nz : 32;
  const long long used = (long long)((nx + kRTX - 1) / kRTX) * ((ny + kRTY - 1) / kRTY) *
                         ((nz + zchunk - 1) / zchunk);
  if (used > cv.tiles) return cudaErrorInvalidValue;  // partial buffer too small
  switch (cv.st.R) {
    case 1: launch_r<T, TL, 1>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 2: launch_r<T, TL, 2>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 3: launch_r<T, TL, 3>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 4: launch_r<T, TL, 4>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 5: launch_r<T, TL, 5>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 6: launch_r<T, TL, 6>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    case 7: launch_r<T, TL, 7>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
    default: launch_r<T, TL, 8>(cv, x, r, pdir, mask, r_lo, p_lo, x_lo, use_df, p_keep, ax, s); break;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t cocg_resid<double, double>(const CocgView<double>&, const cpx<double>*,
                                                cpx<double>*, cpx<double>*, int, cpx<double>*,
                                                cpx<double>*, cpx<double>*, cudaStream_t, bool,
                                                const cpx<double>*, const DfAux*);
template cudaError_t cocg_resid<double, float>(const CocgView<double>&, const cpx<double>*,
                                               cpx<double>*, cpx<double>*, int, cpx<float>*,
                                               cpx<float>*, cpx<float>*, cudaStream_t, bool,
                                               const cpx<float>*, const DfAux*);
template cudaError_t cocg_resid<float, float>(const CocgView<float>&, const cpx<float>*,
                                              cpx<float>*, cpx<float>*, int, cpx<float>*,
                                              cpx<float>*, cpx<float>*, cudaStream_t, bool,
                                               const cpx<float>*, const DfAux*);

}  // namespace rpa
