// Two-point form of the fused COCG direction + H-apply kernel (K_A of the fused iteration,
// Eq. 4 solved by COCG, Section 4), FP32 only, for grids with an even x extent.
//
// Each thread owns two x-adjacent columns of a 64 x 8 tile and walks z like the column-tile
// kernel.  The pair is read and written as one 16-byte vector, the x neighbours of both
// points come from R/2 + 1 aligned 16-byte shared-memory loads (instead of 2R 8-byte loads
// per point), the y neighbours of the pair from one 16-byte load per row, and the index
// arithmetic of a plane is shared by the two points.  The wider tile also shrinks the halo
// per point.  The plane keeps an x offset XO = R rounded up to even so that every pair sits
// on a 16-byte boundary.
#include <cuda_runtime.h>

#include <mutex>

#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kX2TX = 64, kX2TY = 8, kX2Threads = 256;

__device__ __forceinline__ float4 ld4(const cpx<float>* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(cpx<float>* p, const cpx<float>& a, const cpx<float>& b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}

// Where the 2R+1 values of a thread's z window live (ZM):
//   kZRegs   registers, rotated by one plane per step (the original form);
//   kZRing1  a per-thread ring in shared memory (slot = plane mod 2R+1, read at offsets fixed
//            per plane), one centre-plane buffer (two barriers per plane): no register queue,
//            so three blocks fit an SM;
//   kZRing2  the same ring with two centre-plane buffers (one barrier per plane).
// Only the thread that owns a column reads and writes its ring slots, so the ring needs no
// barrier of its own.
constexpr int kZRegs = 0, kZRing1 = 1, kZRing2 = 2;

template <int R>
constexpr size_t x2_ring_bytes() {
  return (size_t)(2 * R + 1) * kX2Threads * sizeof(float4);
}

template <int R, bool FIRST, int ZM>
__global__ void __launch_bounds__(kX2Threads, ZM == kZRing1 ? 3 : 2)
    k_dirmatvec_x2(CocgView<float> cv, FusedBufs<float> fb) {
  using T = float;
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  constexpr bool RING = ZM != kZRegs;
  constexpr int NQ = 2 * R + 1;
  constexpr int XO = R + (R & 1);             // x offset of the tile in the plane (even)
  constexpr int EXN = kX2TX + 2 * XO, EYN = kX2TY + 2 * R;
  constexpr int PLN = EXN * EYN;
  constexpr int NUSED = (kX2TX + 2 * R) * EYN;  // used slots (tile + halo)
  constexpr int NHALO = NUSED - kX2TX * kX2TY;
  constexpr int HPT = (NHALO + kX2Threads - 1) / kX2Threads;
  __shared__ __align__(16) cpx<T> pl[(ZM == kZRing1 ? 1 : 2) * PLN];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float4* ring = reinterpret_cast<float4*>(dyn_smem);  // NQ x kX2Threads (RING)
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int ntx = (nx + kX2TX - 1) / kX2TX;
  const int tx0 = (blockIdx.x % ntx) * kX2TX, ty0 = (blockIdx.x / ntx) * kX2TY;
  const int z0 = blockIdx.z * fb.zchunk, z1 = min(z0 + fb.zchunk, nz);
  const int lx = (threadIdx.x & 31) * 2, ly = threadIdx.x >> 5;
  const int gx = tx0 + lx, gy = ty0 + ly;
  const bool valid = gx < nx && gy < ny;  // nx even: gx + 1 < nx as well
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
  // xy offset of the pair (its first point; -1 outside a Dirichlet boundary)
  int own_xy;
  {
    const int x = wrap_or_neg(gx, nx, st.bcx), y = wrap_or_neg(gy, ny, st.bcy);
    own_xy = (x < 0 || y < 0) ? -1 : x + nx * y;
  }
  // halo elements: R rows above, the 2R padding points of each tile row, R rows below
  int halo_xy[HPT], halo_slot[HPT];
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int hi = threadIdx.x + k * kX2Threads;
    halo_slot[k] = -1;
    halo_xy[k] = -1;
    if (hi < NHALO) {
      constexpr int UX = kX2TX + 2 * R;  // used columns
      int ey, ex;
      if (hi < R * UX) {
        ey = hi / UX;
        ex = hi - ey * UX;
      } else if (hi < R * UX + kX2TY * 2 * R) {
        const int t = hi - R * UX;
        ey = R + t / (2 * R);
        const int c = t - (ey - R) * 2 * R;
        ex = (c < R) ? c : kX2TX + c;
      } else {
        const int t = hi - R * UX - kX2TY * 2 * R;
        ey = R + kX2TY + t / UX;
        ex = t - (ey - R - kX2TY) * UX;
      }
      halo_slot[k] = ey * EXN + ex + (XO - R);
      const int x = wrap_or_neg(tx0 - R + ex, nx, st.bcx), y = wrap_or_neg(ty0 - R + ey, ny, st.bcy);
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
  // pair loads: 16 bytes at an even grid offset when nx is even
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
  constexpr int QL = RING ? 1 : 2 * R + 1;
  cpx<T> za[QL], zb[QL];  // z queues of the two columns (register form)
  // ring slot of plane zz (zz >= z0 - R)
  auto rslot = [&](int zz) -> int { return (zz - z0 + R) % NQ; };
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int zo = zoff(z0 - R + i);
    cpx<T> r0, r1, p0, p1;
    ld2((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, r0, r1, p0, p1);
    const cpx<T> va = comb(r0, p0), vb = comb(r1, p1);
    if constexpr (RING) {
      ring[i * kX2Threads + threadIdx.x] = make_float4(va.re, va.im, vb.re, vb.im);
    } else {
      za[i] = va;
      zb[i] = vb;
    }
  }
  cpx<T> nr0, nr1, np0, np1, h_r[HPT], h_p[HPT];
  auto prefetch = [&](int z) {
    const int zo = zoff(z + R);
    ld2((zo < 0 || own_xy < 0) ? -1 : zo + own_xy, nr0, nr1, np0, np1);
    const int zp = z * plane;
#pragma unroll
    for (int k = 0; k < HPT; ++k) ld1(halo_xy[k] < 0 ? -1 : zp + halo_xy[k], h_r[k], h_p[k]);
  };
  if (z0 < z1) prefetch(z0);
  using A = dacc_t<T>;
  A acc_re = 0, acc_im = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    const int bo = ZM == kZRing1 ? 0 : ((z - z0) & 1) * PLN;
    cpx<T> c, d;  // this column's values at plane z
    int rb = 0;   // ring slot of plane z
    if constexpr (RING) {
      rb = rslot(z);
      const cpx<T> va = comb(nr0, np0), vb = comb(nr1, np1);
      const int sn = rb + R < NQ ? rb + R : rb + R - NQ;  // slot of plane z + R
      ring[sn * kX2Threads + threadIdx.x] = make_float4(va.re, va.im, vb.re, vb.im);
      const float4 cc = ring[rb * kX2Threads + threadIdx.x];
      c = mk<T>(cc.x, cc.y);
      d = mk<T>(cc.z, cc.w);
      if (ZM == kZRing1 && z > z0) __syncthreads();  // everyone is done with plane z - 1
    } else {
      za[2 * R] = comb(nr0, np0);
      zb[2 * R] = comb(nr1, np1);
      c = za[R];
      d = zb[R];
    }
    st4(pl + bo + own_slot, c, d);
#pragma unroll
    for (int k = 0; k < HPT; ++k)
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
      // x: the row segment [own - XO, own + XO + 1] as XO + 1 aligned pairs
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
        if constexpr (RING) {
          const int sl = rb - m >= 0 ? rb - m : rb - m + NQ;
          const int sh_ = rb + m < NQ ? rb + m : rb + m - NQ;
          const float4 lo = ring[sl * kX2Threads + threadIdx.x];
          const float4 hi = ring[sh_ * kX2Threads + threadIdx.x];
          a0 = caxpy_r(a0, st.cz[m], mk<T>(lo.x + hi.x, lo.y + hi.y));
          a1 = caxpy_r(a1, st.cz[m], mk<T>(lo.z + hi.z, lo.w + hi.w));
        } else {
          a0 = caxpy_r(a0, st.cz[m], cadd(za[R - m], za[R + m]));
          a1 = caxpy_r(a1, st.cz[m], cadd(zb[R - m], zb[R + m]));
        }
      }
      st4(w + q, a0, a1);
      st4(pn + q, c, d);
      acc_re += (A)c.re * a0.re - (A)c.im * a0.im + (A)d.re * a1.re - (A)d.im * a1.im;
      acc_im += (A)c.re * a0.im + (A)c.im * a0.re + (A)d.re * a1.im + (A)d.im * a1.re;
    }
    if constexpr (!RING) {
#pragma unroll
      for (int i = 0; i < 2 * R; ++i) {
        za[i] = za[i + 1];
        zb[i] = zb[i + 1];
      }
    }
  }
  A acc2[2] = {acc_re, acc_im};
  __shared__ A sha[8 * 2];
  block_sum_t<A, 2>(acc2, sha);
  if (threadIdx.x == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = (double)acc2[0];
    pp[1] = (double)acc2[1];
  }
}

template <int R, int ZM>
void launch_zm(const CocgView<float>& cv, const FusedBufs<float>& fb, cudaStream_t s) {
  const size_t dyn = ZM == kZRegs ? 0 : x2_ring_bytes<R>();
  const dim3 grid(fb.ntiles_xy, fb.nact, fb.nzchunk);
  if (fb.first)
    k_dirmatvec_x2<R, true, ZM><<<grid, kX2Threads, dyn, s>>>(cv, fb);
  else
    k_dirmatvec_x2<R, false, ZM><<<grid, kX2Threads, dyn, s>>>(cv, fb);
}

template <int R>
void launch_r(const CocgView<float>& cv, const FusedBufs<float>& fb, cudaStream_t s) {
  if (fb.row_ty == kTileX2Ring1)
    launch_zm<R, kZRing1>(cv, fb, s);
  else if (fb.row_ty == kTileX2Ring2)
    launch_zm<R, kZRing2>(cv, fb, s);
  else
    launch_zm<R, kZRegs>(cv, fb, s);
}

// opt-in dynamic shared memory of the ring forms, once per device
cudaError_t x2_attr() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  constexpr int kMax = 96 * 1024;
#define RPA_X2_ATTR(RR, ZZ)                                                                   \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_dirmatvec_x2<RR, true, ZZ>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);             \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_dirmatvec_x2<RR, false, ZZ>,                                  \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
#define RPA_X2_ATTR_R(RR) RPA_X2_ATTR(RR, kZRing1) RPA_X2_ATTR(RR, kZRing2)
  RPA_X2_ATTR_R(1) RPA_X2_ATTR_R(2) RPA_X2_ATTR_R(3) RPA_X2_ATTR_R(4)
  RPA_X2_ATTR_R(5) RPA_X2_ATTR_R(6) RPA_X2_ATTR_R(7) RPA_X2_ATTR_R(8)
#undef RPA_X2_ATTR_R
#undef RPA_X2_ATTR
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

}  // namespace

bool x2_tile_fits(int nx, int R) { return nx % 2 == 0 && R >= 1 && R <= 8; }

int x2_tiles_xy(int nx, int ny) {
  return ((nx + kX2TX - 1) / kX2TX) * ((ny + kX2TY - 1) / kX2TY);
}

cudaError_t launch_dirmatvec_x2_prepare() { return x2_attr(); }

cudaError_t launch_dirmatvec_x2(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                cudaStream_t s) {
  if (fb.row_ty == kTileX2Ring1 || fb.row_ty == kTileX2Ring2) {
    cudaError_t e = x2_attr();
    if (e != cudaSuccess) return e;
  }
  switch (cv.st.R) {
    case 1: launch_r<1>(cv, fb, s); break;
    case 2: launch_r<2>(cv, fb, s); break;
    case 3: launch_r<3>(cv, fb, s); break;
    case 4: launch_r<4>(cv, fb, s); break;
    case 5: launch_r<5>(cv, fb, s); break;
    case 6: launch_r<6>(cv, fb, s); break;
    case 7: launch_r<7>(cv, fb, s); break;
    default: launch_r<8>(cv, fb, s); break;
  }
  return cudaGetLastError();
}

}  // namespace rpa
