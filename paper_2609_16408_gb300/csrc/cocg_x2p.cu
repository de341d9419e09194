// Two-point form of the fused COCG direction + H-apply kernel on packed full rows (K_A of
// the fused iteration, Eq. 4 solved by COCG, Section 4), FP32, stencil radius 6, for grids
// with an even x extent between 26 and 64.
//
// The 64 x 8 two-point tiles leave the lanes past the end of a short row idle (12 of every
// 32 on a 52-point row).  Here a tile is TY full rows: the nx/2 pairs of a row go to
// consecutive threads, row after row, so a 256-thread block holds TY = floor(256 / (nx/2))
// rows and only 256 - TY nx/2 threads own no pair (22 on a 52-point row, against 56 idle
// lanes in the 64 x 8 tiles).  The shared plane keeps the 64 + 2 XO column layout of the
// two-point kernel (compile-time neighbour offsets); the columns past nx + R stay unused.
// Threads that own no pair still load halo values and take part in every barrier.
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kPR = 6;             // stencil radius of this kernel
constexpr int kPThreads = 256;
constexpr int kPMaxX = 64;         // widest row (shared-memory layout)
constexpr int kPMinPairs = 13;     // nx >= 26: at most 19 rows per tile
constexpr int kPHpt = 4;           // halo values per thread (checked on the host)

__device__ __forceinline__ float4 ld4(const cpx<float>* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(cpx<float>* p, const cpx<float>& a, const cpx<float>& b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}

__host__ __device__ constexpr int p_rows(int nx) { return kPThreads / (nx / 2); }

template <bool FIRST, int TY>
__global__ void __launch_bounds__(kPThreads, 2)
    k_dirmatvec_x2p(CocgView<float> cv, FusedBufs<float> fb) {
  using T = float;
  constexpr int R = kPR;
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  constexpr int XO = R + (R & 1);  // x offset of the row start in the plane (even)
  constexpr int EXN = kPMaxX + 2 * XO, EYN = TY + 2 * R;
  constexpr int PLN = EXN * EYN;
  __shared__ __align__(16) cpx<T> pl[2 * PLN];
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int pr = nx >> 1;                   // pairs per row
  const bool owner = (int)threadIdx.x < pr * TY;
  const int lx = owner ? ((int)threadIdx.x % pr) * 2 : 0;
  const int ly = owner ? (int)threadIdx.x / pr : 0;
  const int ty0 = blockIdx.x * TY;
  const int z0 = blockIdx.z * fb.zchunk, z1 = min(z0 + fb.zchunk, nz);
  const int gx = lx, gy = ty0 + ly;
  const bool valid = owner && gy < ny;
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
  // xy offset of the owned pair (its first point; -1 outside a Dirichlet boundary); rows past
  // ny hold the wrapped rows that the last rows of the grid need as y neighbours
  int own_xy = -1;
  if (owner) {
    const int y = wrap_or_neg(gy, ny, st.bcy);
    own_xy = y < 0 ? -1 : gx + nx * y;
  }
  // halo: R rows above and below (columns x in [-R, nx + R)) and R columns on either side
  // of the TY owned rows
  const int ux = nx + 2 * R;
  const int nhalo = 2 * R * ux + TY * 2 * R;
  int halo_xy[kPHpt], halo_slot[kPHpt];
#pragma unroll
  for (int k = 0; k < kPHpt; ++k) {
    const int hi = threadIdx.x + k * kPThreads;
    halo_slot[k] = -1;
    halo_xy[k] = -1;
    if (hi < nhalo) {
      int ey, ex;  // row in the plane, column counted from x = -R
      if (hi < R * ux) {
        ey = hi / ux;
        ex = hi - ey * ux;
      } else if (hi < R * ux + TY * 2 * R) {
        const int t = hi - R * ux;
        ey = R + t / (2 * R);
        const int c = t - (ey - R) * 2 * R;
        ex = (c < R) ? c : nx + c;
      } else {
        const int t = hi - R * ux - TY * 2 * R;
        ey = R + TY + t / ux;
        ex = t - (ey - R - TY) * ux;
      }
      halo_slot[k] = ey * EXN + ex + (XO - R);
      const int x = wrap_or_neg(ex - R, nx, st.bcx), y = wrap_or_neg(ty0 - R + ey, ny, st.bcy);
      halo_xy[k] = (x < 0 || y < 0) ? -1 : x + nx * y;
    }
  }
  const int own_slot = (ly + R) * EXN + lx + XO;  // even
  auto zoff = [&](int z) -> int {
    const int zz = wrap_or_neg(z, nz, st.bcz);
    return zz < 0 ? -1 : zz * plane;
  };
  auto comb = [&](const cpx<T>& rv, const cpx<T>& pv) -> cpx<T> {
    if (FIRST) return rv;
    return cadd(rv, cmul(be, pv));
  };
  auto ld2 = [&](int q, cpx<T>& r0, cpx<T>& r1, cpx<T>& p0, cpx<T>& p1) {
    if (q < 0) {
      r0 = r1 = p0 = p1 = mk<T>((T)0, (T)0);
    } else {
      const float4 a = ld4(r + q);
      r0 = mk<T>(a.x, a.y);
      r1 = mk<T>(a.z, a.w);
      if (!FIRST) {
        const float4 c = ld4(po + q);
        p0 = mk<T>(c.x, c.y);
        p1 = mk<T>(c.z, c.w);
      }
    }
  };
  auto ld1 = [&](int q, cpx<T>& rv, cpx<T>& pv) {
    if (q < 0) {
      rv = mk<T>((T)0, (T)0);
      pv = rv;
    } else {
      rv = r[q];
      if (!FIRST) pv = po[q];
    }
  };
  cpx<T> za[2 * R + 1], zb[2 * R + 1];  // z queues of the two columns
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    cpx<T> r0, r1, p0, p1;
    ld2((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, r0, r1, p0, p1);
    za[i] = comb(r0, p0);
    zb[i] = comb(r1, p1);
  }
  cpx<T> nr0, nr1, np0, np1, h_r[kPHpt], h_p[kPHpt];
  auto prefetch = [&](int z) {
    const int zo = zoff(z + R);
    ld2((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, nr0, nr1, np0, np1);
    const int zp = z * plane;
#pragma unroll
    for (int k = 0; k < kPHpt; ++k) ld1(halo_xy[k] < 0 ? -1 : zp + halo_xy[k], h_r[k], h_p[k]);
  };
  if (z0 < z1) prefetch(z0);
  using A = dacc_t<T>;
  A acc_re = 0, acc_im = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    const int bo = ((z - z0) & 1) * PLN;
    za[2 * R] = comb(nr0, np0);
    zb[2 * R] = comb(nr1, np1);
    const cpx<T> c = za[R], d = zb[R];  // this pair's values at plane z
    if (owner) st4(pl + bo + own_slot, c, d);
#pragma unroll
    for (int k = 0; k < kPHpt; ++k)
      if (halo_slot[k] >= 0) pl[bo + halo_slot[k]] = comb(h_r[k], h_p[k]);
    if (z + 1 < z1) prefetch(z + 1);  // in flight while this plane is computed
    __syncthreads();
    if (valid) {
      const int q = own_xy + z * plane;
      const cpx<T>* cs = pl + bo + own_slot;
      const float2 vv = *reinterpret_cast<const float2*>(vloc + q);  // q even: 8-byte aligned
      const T dg0 = c0 + vv.x, dg1 = c0 + vv.y;
      cpx<T> a0 = mk<T>(dg0 * c.re - (sigma.re * c.re - sigma.im * c.im),
                        dg0 * c.im - (sigma.re * c.im + sigma.im * c.re));
      cpx<T> a1 = mk<T>(dg1 * d.re - (sigma.re * d.re - sigma.im * d.im),
                        dg1 * d.im - (sigma.re * d.im + sigma.im * d.re));
      cpx<T> xr[2 * XO + 2];
#pragma unroll
      for (int k = 0; k <= XO; ++k) {
        const float4 v = ld4(cs - XO + 2 * k);
        xr[2 * k] = mk<T>(v.x, v.y);
        xr[2 * k + 1] = mk<T>(v.z, v.w);
      }
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        a0 = caxpy_r(a0, st.cx[m], cadd(xr[XO - m], xr[XO + m]));
        a1 = caxpy_r(a1, st.cx[m], cadd(xr[XO + 1 - m], xr[XO + 1 + m]));
        const float4 up = ld4(cs - m * EXN), dn = ld4(cs + m * EXN);
        a0 = caxpy_r(a0, st.cy[m], mk<T>(up.x + dn.x, up.y + dn.y));
        a1 = caxpy_r(a1, st.cy[m], mk<T>(up.z + dn.z, up.w + dn.w));
        a0 = caxpy_r(a0, st.cz[m], cadd(za[R - m], za[R + m]));
        a1 = caxpy_r(a1, st.cz[m], cadd(zb[R - m], zb[R + m]));
      }
      st4(w + q, a0, a1);
      st4(pn + q, c, d);
      acc_re += (A)c.re * a0.re - (A)c.im * a0.im + (A)d.re * a1.re - (A)d.im * a1.im;
      acc_im += (A)c.re * a0.im + (A)c.im * a0.re + (A)d.re * a1.im + (A)d.im * a1.re;
    }
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
      za[i] = za[i + 1];
      zb[i] = zb[i + 1];
    }
  }
  A acc2[2] = {acc_re, acc_im};
  __shared__ A sha[(kPThreads / 32) * 2];
  block_sum_t<A, 2>(acc2, sha);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = (double)acc2[0];
    pp[1] = (double)acc2[1];
  }
}

template <int TY>
void launch_ty(const CocgView<float>& cv, const FusedBufs<float>& fb, cudaStream_t s) {
  const dim3 grid(fb.ntiles_xy, fb.nact, fb.nzchunk);
  if (fb.first)
    k_dirmatvec_x2p<true, TY><<<grid, kPThreads, 0, s>>>(cv, fb);
  else
    k_dirmatvec_x2p<false, TY><<<grid, kPThreads, 0, s>>>(cv, fb);
}

}  // namespace

bool x2p_tile_fits(int nx, int R) {
  if (R != kPR || nx % 2 != 0 || nx > kPMaxX || nx / 2 < kPMinPairs) return false;
  const int ty = p_rows(nx);
  return 2 * R * (nx + 2 * R) + ty * 2 * R <= kPHpt * kPThreads;  // halo values fit
}

int x2p_tiles_xy(int nx, int ny) {
  const int ty = p_rows(nx);
  return (ny + ty - 1) / ty;
}

cudaError_t launch_dirmatvec_x2p(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                 cudaStream_t s) {
  if (!x2p_tile_fits(cv.st.nx, cv.st.R)) return cudaErrorInvalidValue;
  switch (p_rows(cv.st.nx)) {
    case 8: launch_ty<8>(cv, fb, s); break;
    case 9: launch_ty<9>(cv, fb, s); break;
    case 10: launch_ty<10>(cv, fb, s); break;
    case 11: launch_ty<11>(cv, fb, s); break;
    case 12: launch_ty<12>(cv, fb, s); break;
    case 13: launch_ty<13>(cv, fb, s); break;
    case 14: launch_ty<14>(cv, fb, s); break;
    case 15: launch_ty<15>(cv, fb, s); break;
    case 16: launch_ty<16>(cv, fb, s); break;
    case 17: launch_ty<17>(cv, fb, s); break;
    case 18: launch_ty<18>(cv, fb, s); break;
    case 19: launch_ty<19>(cv, fb, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rpa
