// Band form of the fused COCG direction + H-apply kernel (K_A of the fused iteration, Eq. 4
// solved by COCG, Section 4), FP32, for grids with an even x extent of at most 64 points.
//
// A block owns a band of TY complete x rows of one system (TY divides ny) and walks along z.
// Each thread owns two x-adjacent points (one 16-byte pair), as in the two-point tile kernel.
// What differs:
//  * Full rows: on a 52- or 40-point x axis no lane falls outside the grid, and the halo is
//    only the R rows above and below the band -- the x wrap of a periodic axis is written
//    into padding slots of the shared plane by the threads that own the edge pairs, so no x
//    halo is loaded at all.
//  * Inputs arrive through a D-stage cp.async pipeline instead of register prefetch: at plane
//    z a stage carries the band's own pairs of plane z + R (they enter the per-thread register
//    queue of the z direction) and the halo rows of plane z (the centre of the stencil).
//    Several planes of loads are in flight without holding registers.  Every thread reads back
//    only the stage slots it copied itself, so a stage needs no barrier; one barrier per plane
//    publishes the centre plane.
//  * Every stencil neighbour is read at a compile-time offset from the thread's own slot (the
//    shared rows have a fixed pitch of 64 + 2 XO pairs' worth of points).
// Out-of-range rows and planes of a Dirichlet axis are zero-filled by the copy itself
// (source size 0).
#include <cuda_runtime.h>

#include <mutex>

#include "cocg.cuh"
#include "cocg_fused.cuh"
#include "fused_dev.cuh"

namespace rpa {

namespace {

constexpr int kBandStages = 3;
constexpr int kBandMaxThreads = 704;   // 22 warps
constexpr int kBandSmallThreads = 352;
constexpr int kBandMaxHalo = 2;        // halo pairs copied per thread and plane
constexpr size_t kBandSmemMax = 200 * 1024;

__device__ __forceinline__ float4 ld4(const cpx<float>* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(cpx<float>* p, const cpx<float>& a, const cpx<float>& b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}
// 16-byte asynchronous copy global -> shared; src_size 0 writes zeros and reads nothing
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int R>
__host__ __device__ constexpr int band_xo() {
  return R + (R & 1);
}
template <int R>
__host__ __device__ constexpr int band_pitch() {
  return 64 + 2 * band_xo<R>();
}

// dynamic shared memory of one block: two centre planes and D stages
size_t band_smem(int nx, int R, int ty) {
  const int xo = R + (R & 1), pitch = 64 + 2 * xo;
  const size_t centre = 2 * sizeof(cpx<float>) * (size_t)(ty + 2 * R) * pitch;
  const size_t stage = (size_t)kBandStages * 2 * sizeof(float4) *
                       ((size_t)ty * (nx / 2) + (size_t)2 * R * (nx / 2));
  return centre + stage;
}

template <int R, bool FIRST, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_dirmatvec_band(CocgView<float> cv, FusedBufs<float> fb) {
  using T = float;
  using A = dacc_t<T>;
  const int s = cv.list ? cv.list[blockIdx.y] : blockIdx.y;
  if (s < 0 || cv.sysi[(long long)s * kSysI + kStatus] != kActive) return;
  constexpr int XO = band_xo<R>();
  constexpr int PITCH = band_pitch<R>();
  constexpr int D = kBandStages;
  const Stencil<T>& st = cv.st;
  const int nx = st.nx, ny = st.ny, nz = st.nz;
  const int plane = nx * ny;
  const int TY = fb.band_ty, PPR = nx >> 1;
  const int nown = TY * PPR, nhal = 2 * R * PPR;  // pairs of the band and of its halo rows
  const int PLN = (TY + 2 * R) * PITCH;           // complex slots of one centre plane
  const int SSTR = 2 * (nown + nhal);             // float4 slots of one stage
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  cpx<T>* cbuf = reinterpret_cast<cpx<T>*>(dyn_smem);
  float4* stg = reinterpret_cast<float4*>(cbuf + 2 * PLN);
  __shared__ A sha[32 * 2];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int y0 = blockIdx.x * TY;
  const int z0 = blockIdx.z * fb.zchunk, z1 = min(z0 + fb.zchunk, nz);
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
  // x padding of every row of both centre planes: zero once (a Dirichlet x axis keeps the
  // zeros; on a periodic axis the owners of the edge pairs overwrite them every plane)
  for (int i = tid; i < 2 * (TY + 2 * R) * 2 * XO; i += nthr) {
    const int row = i / (2 * XO), c = i - row * (2 * XO);
    const int x = c < XO ? c : nx + c;  // slots [0, XO) and [XO + nx, nx + 2 XO)
    cbuf[row * PITCH + x] = mk<T>((T)0, (T)0);
  }
  const bool perx = st.bcx == 0;
  // own pair
  const bool own = tid < nown;
  const int ly = own ? tid / PPR : 0;
  const int gx = own ? 2 * (tid - ly * PPR) : 0;
  const int own_xy = gx + nx * (y0 + ly);
  const int own_slot = (ly + R) * PITCH + XO + gx;
  const bool own_wp = perx && gx < XO;        // copy also at x + nx (right padding)
  const bool own_wm = perx && gx >= nx - XO;  // copy also at x - nx (left padding)
  // halo pairs: rows y0 - R .. y0 - 1 and y0 + TY .. y0 + TY + R - 1 of the centre plane
  // (the stencil is a star: halo rows are read only above and below the band's own points,
  // so they need no x padding)
  int hal_xy[kBandMaxHalo], hal_slot[kBandMaxHalo];
#pragma unroll
  for (int k = 0; k < kBandMaxHalo; ++k) {
    const int h = tid + k * nthr;
    hal_slot[k] = -1;
    hal_xy[k] = -1;
    if (h < nhal) {
      const int hr = h / PPR, hx = 2 * (h - hr * PPR);
      const int lr = hr < R ? hr : TY + hr;  // row of the centre plane buffer
      const int yy = wrap_or_neg(y0 - R + lr, ny, st.bcy);
      hal_xy[k] = yy < 0 ? -1 : hx + nx * yy;
      hal_slot[k] = lr * PITCH + XO + hx;
    }
  }
  auto zoff = [&](int z) -> int {
    const int zz = wrap_or_neg(z, nz, st.bcz);
    return zz < 0 ? -1 : zz * plane;
  };
  auto comb = [&](T rr, T ri, T pr, T pi) -> cpx<T> {
    if (FIRST) return mk<T>(rr, ri);
    return mk<T>(rr + be.re * pr - be.im * pi, ri + be.re * pi + be.im * pr);
  };
  // stage of plane zi: own pairs of plane zi + R and halo pairs of plane zi
  auto issue = [&](int zi) {
    if (zi < z1) {
      float4* sb = stg + ((zi - z0) % D) * SSTR;
      if (own) {
        const int zo = zoff(zi + R);
        const bool v = zo >= 0;
        const int q = v ? zo + own_xy : 0;
        cp_async16(sb + 2 * tid, r + q, v);
        if (!FIRST) cp_async16(sb + 2 * tid + 1, po + q, v);
      }
      const int zp = zi * plane;
#pragma unroll
      for (int k = 0; k < kBandMaxHalo; ++k) {
        if (hal_slot[k] < 0) continue;
        const bool v = hal_xy[k] >= 0;
        const int q = v ? zp + hal_xy[k] : 0;
        const int j = nown + tid + k * nthr;
        cp_async16(sb + 2 * j, r + q, v);
        if (!FIRST) cp_async16(sb + 2 * j + 1, po + q, v);
      }
    }
    cp_async_commit();  // one group per plane, empty past the chunk
  };
#pragma unroll
  for (int i = 0; i < D - 1; ++i) issue(z0 + i);
  // z queues of the two points: planes z0 - R .. z0 + R - 1 now, z0 + R from the first stage
  cpx<T> za[2 * R + 1], zb[2 * R + 1];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    za[i] = zb[i] = mk<T>((T)0, (T)0);
    const int zo = zoff(z0 - R + i);
    if (own && zo >= 0) {
      const float4 a = ld4(r + zo + own_xy);
      float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!FIRST) c = ld4(po + zo + own_xy);
      za[i] = comb(a.x, a.y, c.x, c.y);
      zb[i] = comb(a.z, a.w, c.z, c.w);
    }
  }
  A acc_re = 0, acc_im = 0;
  const T c0 = st.c0;
  for (int z = z0; z < z1; ++z) {
    cp_async_wait<D - 2>();  // this thread's copies of plane z have landed
    issue(z + D - 1);
    const float4* sb = stg + ((z - z0) % D) * SSTR;
    cpx<T>* cb = cbuf + ((z - z0) & 1) * PLN;
    if (own) {
      const float4 a = sb[2 * tid];
      const float4 c = FIRST ? make_float4(0.f, 0.f, 0.f, 0.f) : sb[2 * tid + 1];
      za[2 * R] = comb(a.x, a.y, c.x, c.y);
      zb[2 * R] = comb(a.z, a.w, c.z, c.w);
      st4(cb + own_slot, za[R], zb[R]);
      if (own_wp) st4(cb + own_slot + nx, za[R], zb[R]);
      if (own_wm) st4(cb + own_slot - nx, za[R], zb[R]);
    }
#pragma unroll
    for (int k = 0; k < kBandMaxHalo; ++k) {
      if (hal_slot[k] < 0) continue;
      const int j = nown + tid + k * nthr;
      const float4 a = sb[2 * j];
      const float4 c = FIRST ? make_float4(0.f, 0.f, 0.f, 0.f) : sb[2 * j + 1];
      st4(cb + hal_slot[k], comb(a.x, a.y, c.x, c.y), comb(a.z, a.w, c.z, c.w));
    }
    __syncthreads();
    if (own) {
      const int q = own_xy + z * plane;
      const cpx<T> c = za[R], d = zb[R];
      const cpx<T>* cs = cb + own_slot;
      const float2 vv = *reinterpret_cast<const float2*>(vloc + q);  // q even: 8-byte aligned
      const T dg0 = c0 + vv.x, dg1 = c0 + vv.y;
      cpx<T> a0 = mk<T>(dg0 * c.re - (sigma.re * c.re - sigma.im * c.im),
                        dg0 * c.im - (sigma.re * c.im + sigma.im * c.re));
      cpx<T> a1 = mk<T>(dg1 * d.re - (sigma.re * d.re - sigma.im * d.im),
                        dg1 * d.im - (sigma.re * d.im + sigma.im * d.re));
      // x neighbours: the XO + 1 aligned pairs of the row segment [own - XO, own + XO + 1],
      // each added to both points as soon as it is loaded (offsets are compile-time)
#pragma unroll
      for (int k = 0; k <= XO; ++k) {
        const float4 v = ld4(cs - XO + 2 * k);
        const cpx<T> va = mk<T>(v.x, v.y), vb = mk<T>(v.z, v.w);
        const int da = 2 * k - XO, db = da + 1;  // offsets from the first point
        if (da != 0 && da >= -R && da <= R) a0 = caxpy_r(a0, st.cx[da < 0 ? -da : da], va);
        if (db != 0 && db >= -R && db <= R) a0 = caxpy_r(a0, st.cx[db < 0 ? -db : db], vb);
        if (da != 1 && da - 1 >= -R && da - 1 <= R)
          a1 = caxpy_r(a1, st.cx[da - 1 < 0 ? 1 - da : da - 1], va);
        if (db != 1 && db - 1 >= -R && db - 1 <= R)
          a1 = caxpy_r(a1, st.cx[db - 1 < 0 ? 1 - db : db - 1], vb);
      }
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float4 up = ld4(cs - m * PITCH), dn = ld4(cs + m * PITCH);
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
  cp_async_wait<0>();  // nothing may land after the block has exited
  A acc2[2] = {acc_re, acc_im};
  block_sum_t<A, 2>(acc2, sha);
  if (tid == 0) {
    const int pid = blockIdx.x + gridDim.x * blockIdx.z;
    double* pp = cv.part + ((long long)s * cv.tiles + pid) * 4;
    pp[0] = (double)acc2[0];
    pp[1] = (double)acc2[1];
  }
}

template <int R>
void launch_r(const CocgView<float>& cv, const FusedBufs<float>& fb, cudaStream_t s) {
  const int ty = fb.band_ty;
  const int thr = ((ty * (cv.st.nx / 2) + 31) / 32) * 32;
  const size_t smem = band_smem(cv.st.nx, R, ty);
  const dim3 grid(cv.st.ny / ty, fb.nact, fb.nzchunk);
  if (thr <= kBandSmallThreads) {
    if (fb.first)
      k_dirmatvec_band<R, true, kBandSmallThreads><<<grid, thr, smem, s>>>(cv, fb);
    else
      k_dirmatvec_band<R, false, kBandSmallThreads><<<grid, thr, smem, s>>>(cv, fb);
  } else {
    if (fb.first)
      k_dirmatvec_band<R, true, kBandMaxThreads><<<grid, thr, smem, s>>>(cv, fb);
    else
      k_dirmatvec_band<R, false, kBandMaxThreads><<<grid, thr, smem, s>>>(cv, fb);
  }
}

// opt-in dynamic shared memory of the band kernels, once per device
cudaError_t band_attr() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
#define RPA_BAND_ATTR(RR)                                                                     \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_dirmatvec_band<RR, true, kBandSmallThreads>,                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemMax);      \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_dirmatvec_band<RR, false, kBandSmallThreads>,                  \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemMax);      \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_dirmatvec_band<RR, true, kBandMaxThreads>,                     \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemMax);      \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_dirmatvec_band<RR, false, kBandMaxThreads>,                    \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemMax);
  RPA_BAND_ATTR(1) RPA_BAND_ATTR(2) RPA_BAND_ATTR(3) RPA_BAND_ATTR(4)
  RPA_BAND_ATTR(5) RPA_BAND_ATTR(6) RPA_BAND_ATTR(7) RPA_BAND_ATTR(8)
#undef RPA_BAND_ATTR
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

}  // namespace

bool band_tile_fits(int nx, int ny, int R, int ty, int ngroup) {
  if (nx % 2 != 0 || nx > 64 || R < 1 || R > 8 || nx < R + (R & 1)) return false;
  if (ty < 1 || ty > ny || ny % ty != 0) return false;
  const int thr = ((ty * (nx / 2) + 31) / 32) * 32;
  if (thr < 64 || thr > kBandMaxThreads) return false;
  if (2 * R * (nx / 2) > kBandMaxHalo * thr) return false;  // halo pairs per thread
  (void)ngroup;
  return band_smem(nx, R, ty) <= kBandSmemMax;
}

int band_candidates(int nx, int ny, int R, int ngroup, int* out, int maxn) {
  int cnt = 0;
  for (int ty = 1; ty <= ny && cnt < maxn; ++ty) {
    if (!band_tile_fits(nx, ny, R, ty, ngroup)) continue;
    const int thr = ty * (nx / 2);
    if (thr < 160) continue;  // too few warps per block to hide the plane barrier
    out[cnt++] = ty;
  }
  return cnt;
}

cudaError_t launch_dirmatvec_band_prepare() { return band_attr(); }

cudaError_t launch_dirmatvec_band(const CocgView<float>& cv, const FusedBufs<float>& fb,
                                  cudaStream_t s) {
  if (!band_tile_fits(cv.st.nx, cv.st.ny, cv.st.R, fb.band_ty, cv.nl.ngroup))
    return cudaErrorInvalidValue;
  cudaError_t e = band_attr();
  if (e != cudaSuccess) return e;
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
