// Galerkin projection over the occupied space (Section 4) on the 5th-generation tensor cores
// (tcgen05, kind::tf32) for the mixed form:
//   G_b = Psi diag(u_b) Psi^T             (k_gram_tc: M = N = 128 state tiles, K = points)
//   x0_{b,n}(r) = sum_k psi_k(r) C_b[k][n]  (k_x0_tc: M = 128 points, N = 2 N_s (re, im),
//                                            K = states)
// Operands are staged by the block's threads into shared memory in the K-major core-matrix
// layout (8 rows x 16 bytes, no swizzle); one thread issues tcgen05.mma, accumulating in TMEM;
// tcgen05.commit arrives on an mbarrier; the epilogue reads TMEM with tcgen05.ld.
// Operand forms (template flag BF16):
//   * TF32x3 (default mixed form): each fp32 operand is split into tf32 hi + lo parts and the
//     product is formed as hi*hi + hi*lo + lo*hi, which keeps the result at fp32 level (a
//     single tf32 pass would leave ~5e-4 relative error in the occupied-space projection).
//   * BF16 (kind::f16, bf16 A and B, f32 accumulation): one pass on operands rounded to bf16
//     (8-bit significand, relative rounding 2^-9).  The guess is then accurate to ~1e-2
//     relative; COCG removes the difference, at the cost of some extra iterations.
// Both forms use the same byte layout: a stage holds 128 bytes of K per row (32 tf32 or
// 64 bf16).  Every mbarrier wait is bounded, and the block takes each wait's outcome
// together (__syncthreads_and), so that all threads leave the pipeline at the same step.  On
// expiry the kernel records an error code, waits (bounded, full limit) for the commit of the
// last stage it issued -- which covers every MMA in flight -- frees TMEM and returns.  With
// test_expire the first pipeline wait is made on a barrier nothing arrives on, with a short
// limit, before any MMA is issued: the failure path can then be exercised without a fault.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cocg.cuh"
#include "umma.cuh"

namespace rpa {

namespace {
constexpr int kTK = 32;                       // tf32 K elements per shared-memory stage
constexpr int kTK16 = 64;                     // bf16 K elements per stage (same bytes)
constexpr uint32_t kTileBytes128 = 128 * kTK * 4;  // 128 rows x 128 bytes
constexpr uint32_t kWaitLimit = 1u << 26;
constexpr uint32_t kTestWaitLimit = 1u << 10;  // polls of the test_expire wait

// byte offset of (row, k) in a K-major tile of 32 tf32 per row (core matrices 8 x 16 B;
// LBO = 128 B between K-adjacent core matrices, SBO = 1024 B between 8-row groups)
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return ((uint32_t)(row >> 3) << 10) + ((uint32_t)(k >> 2) << 7) + ((uint32_t)(row & 7) << 4) +
         ((uint32_t)(k & 3) << 2);
}
constexpr uint32_t kLBO = 128, kSBO = 1024;
// the same layout for 16-bit elements (8 per core-matrix row)
__device__ __forceinline__ uint32_t kmaj16(int row, int k) {
  return ((uint32_t)(row >> 3) << 10) + ((uint32_t)(k >> 3) << 7) + ((uint32_t)(row & 7) << 4) +
         ((uint32_t)(k & 7) << 1);
}

__device__ __forceinline__ void put_bf16(uint8_t* t, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(t + off) = __float2bfloat16_rn(v);
}

// one bf16 MMA per 16-wide K step over a 64-wide stage
__device__ __forceinline__ void issue_stage_bf16(uint32_t tmem, uint32_t a, uint32_t b,
                                                 uint32_t idesc, bool first) {
#pragma unroll
  for (int kk = 0; kk < kTK16; kk += 16) {
    const uint32_t o = (uint32_t)kk * 16;  // 2 core matrices (16 bf16) along K
    umma::mma_bf16(tmem, umma::smem_desc(a + o, kLBO, kSBO), umma::smem_desc(b + o, kLBO, kSBO),
                   idesc, (first && kk == 0) ? 0u : 1u);
  }
}

__device__ __forceinline__ void put_split(uint8_t* hi, uint8_t* lo, uint32_t off, float v) {
  const float h = umma::to_tf32(v);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = umma::to_tf32(v - h);
}

// three tf32 MMAs (hi*hi + hi*lo + lo*hi) over one 32-wide K stage
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t ahi, uint32_t alo, uint32_t bhi,
                                            uint32_t blo, uint32_t idesc, bool first) {
#pragma unroll
  for (int kk = 0; kk < kTK; kk += 8) {
    const uint32_t o = (uint32_t)kk * 32;  // 2 core matrices (8 tf32) along K
    const uint64_t dah = umma::smem_desc(ahi + o, kLBO, kSBO);
    const uint64_t dal = umma::smem_desc(alo + o, kLBO, kSBO);
    const uint64_t dbh = umma::smem_desc(bhi + o, kLBO, kSBO);
    const uint64_t dbl = umma::smem_desc(blo + o, kLBO, kSBO);
    umma::mma_tf32(tmem, dah, dbh, idesc, (first && kk == 0) ? 0u : 1u);
    umma::mma_tf32(tmem, dah, dbl, idesc, 1u);
    umma::mma_tf32(tmem, dal, dbh, idesc, 1u);
  }
}
}  // namespace

// gpart[b][c][k][n] = sum_{r in chunk c} psi_k(r) psi_n(r) u_b(r) for one 128 x 128 tile.
// Dynamic shared memory: 2 stages x (A_hi, A_lo, B_hi, B_lo) x 16 KB = 128 KB (TF32x3), or
// 2 stages x (A, B) x 16 KB = 64 KB (BF16).
template <bool BF16>
__global__ void __launch_bounds__(128, 1)
    k_gram_tc(long long nd, int ns, const float* __restrict__ psi, const float* __restrict__ u,
              const int* __restrict__ active, int nchunk, long long chunk_len, int ntile_n,
              int nN, double* __restrict__ gpart, int* __restrict__ err, int test_expire) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[3];  // [2]: test_expire only, never arrived on
  __shared__ uint32_t tmem_base;
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int kt = blockIdx.x / ntile_n, nt = blockIdx.x - kt * ntile_n;
  const int k0 = kt * 128, n0 = nt * 128;
  const int c = blockIdx.z;
  const long long r0 = (long long)c * chunk_len;
  const long long r1 = min(r0 + chunk_len, nd);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mb0 = umma::smem_addr(&mbar[0]), mb1 = umma::smem_addr(&mbar[1]);
  const uint32_t mbx = umma::smem_addr(&mbar[2]);
  if (warp == 0) {
    umma::tmem_alloc(umma::smem_addr(&tmem_base), 128);
    umma::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    umma::mbar_init(mb0, 1);
    umma::mbar_init(mb1, 1);
    umma::mbar_init(mbx, 1);
    umma::mbar_fence_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = BF16 ? umma::idesc_bf16(128, nN) : umma::idesc_tf32(128, nN);
  const float* ub = u + (long long)b * nd;
  const long long span = r1 > r0 ? r1 - r0 : 0;
  constexpr int TK = BF16 ? kTK16 : kTK;
  const int nsteps = (int)((span + TK - 1) / TK);
  bool ok = true;
  int issued = 0;  // stages whose MMAs were issued and committed (block-uniform)
  for (int step = 0; step < nsteps; ++step) {
    const int st = step & 1;
    if (step >= 2 || (test_expire && step == 0)) {
      const bool w = (test_expire && step == 0)
                         ? umma::mbar_wait_bounded(mbx, 0, kTestWaitLimit)
                         : umma::mbar_wait_bounded(st ? mb1 : mb0, ((step - 2) >> 1) & 1,
                                                   kWaitLimit);
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    uint8_t* ahi = smem + st * (BF16 ? 2 : 4) * kTileBytes128;
    uint8_t* alo = ahi + kTileBytes128;
    uint8_t* bhi = BF16 ? alo : alo + kTileBytes128;
    uint8_t* blo = bhi + kTileBytes128;
    const long long rb = r0 + (long long)step * TK;
    for (int e = threadIdx.x; e < 128 * TK; e += 128) {
      const int row = e / TK, kk = e - row * TK;
      const long long r = rb + kk;
      const bool vr = r < r1;
      const int k = k0 + row, n = n0 + row;
      const float a = (vr && k < ns) ? psi[(long long)k * nd + r] : 0.f;
      const float bv = (vr && n < ns) ? psi[(long long)n * nd + r] * ub[r] : 0.f;
      if (BF16) {
        const uint32_t off = kmaj16(row, kk);
        put_bf16(ahi, off, a);
        put_bf16(bhi, off, bv);
      } else {
        const uint32_t off = kmaj(row, kk);
        put_split(ahi, alo, off, a);
        put_split(bhi, blo, off, bv);
      }
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma::fence_after_sync();
      if (BF16)
        issue_stage_bf16(tmem, umma::smem_addr(ahi), umma::smem_addr(bhi), idesc, step == 0);
      else
        issue_stage(tmem, umma::smem_addr(ahi), umma::smem_addr(alo), umma::smem_addr(bhi),
                    umma::smem_addr(blo), idesc, step == 0);
      umma::mma_commit(st ? mb1 : mb0);
    }
    issued = step + 1;
  }
  if (issued > 0) {  // the last issued commit covers every MMA issued before it
    const int last = issued - 1;
    const bool done = umma::mbar_wait_bounded((last & 1) ? mb1 : mb0, (last >> 1) & 1, kWaitLimit);
    ok = ok && done;
  }
  ok = __syncthreads_and(ok) != 0;
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  umma::fence_after_sync();
  double* out = gpart + ((long long)b * nchunk + c) * ns * ns;
  const int k = k0 + warp * 32 + lane;
  for (int j0 = 0; j0 < nN; j0 += 16) {
    float v[16];
    if (issued > 0 && ok) {
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int n = n0 + j0 + i;
      if (k < ns && n < ns) out[(long long)k * ns + n] = (double)v[i];
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 128);
}

// x0[(b,n)][r] = sum_k psi_k(r) C_b[k][n] for a 128-point tile and 128 states (N = 256
// columns: re, im interleaved).  Dynamic shared memory, one stage: A_hi, A_lo (128 rows) and
// B_hi, B_lo (256 rows) of 128 bytes each, 96 KB (TF32x3); A and B only, 48 KB (BF16).
template <bool BF16>
__global__ void __launch_bounds__(128, 1)
    k_x0_tc(long long nd, int ns, const float* __restrict__ psi, const cpx<float>* __restrict__ cmat,
            const int* __restrict__ active, int ntile_n, int nN, cpx<float>* __restrict__ x0,
            int* __restrict__ err, int test_expire) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];  // [1]: test_expire only, never arrived on
  __shared__ uint32_t tmem_base;
  const int b = blockIdx.y / ntile_n, nt = blockIdx.y - b * ntile_n;
  if (active && !active[b]) return;
  const long long r0 = (long long)blockIdx.x * 128;
  const int n0 = nt * 128;  // states n0 .. n0+127 -> columns 2(n - n0) + {0, 1}
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mb = umma::smem_addr(&mbar[0]), mbx = umma::smem_addr(&mbar[1]);
  if (warp == 0) {
    umma::tmem_alloc(umma::smem_addr(&tmem_base), 256);
    umma::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    umma::mbar_init(mb, 1);
    umma::mbar_init(mbx, 1);
    umma::mbar_fence_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = BF16 ? umma::idesc_bf16(128, nN) : umma::idesc_tf32(128, nN);
  constexpr int TK = BF16 ? kTK16 : kTK;
  uint8_t* ahi = smem;
  uint8_t* alo = ahi + kTileBytes128;
  uint8_t* bhi = BF16 ? alo : alo + kTileBytes128;
  uint8_t* blo = bhi + 2 * kTileBytes128;
  const cpx<float>* cb = cmat + (long long)b * ns * ns;
  const int nsteps = (ns + TK - 1) / TK;
  bool ok = true;
  int issued = 0;  // stages whose MMAs were issued and committed (block-uniform)
  for (int step = 0; step < nsteps; ++step) {
    if (step >= 1 || test_expire) {
      const bool w = (test_expire && step == 0)
                         ? umma::mbar_wait_bounded(mbx, 0, kTestWaitLimit)
                         : umma::mbar_wait_bounded(mb, (step - 1) & 1, kWaitLimit);
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    const int kb = step * TK;
    for (int e = threadIdx.x; e < 128 * TK; e += 128) {
      const int kk = e >> 7, row = e & 127;  // consecutive threads: consecutive points
      const long long r = r0 + row;
      const float a = (r < nd && kb + kk < ns) ? psi[(long long)(kb + kk) * nd + r] : 0.f;
      if (BF16)
        put_bf16(ahi, kmaj16(row, kk), a);
      else
        put_split(ahi, alo, kmaj(row, kk), a);
    }
    for (int e = threadIdx.x; e < 256 * TK; e += 128) {
      const int kk = e >> 8, j = e & 255;
      const int n = n0 + (j >> 1);
      float v = 0.f;
      if (kb + kk < ns && n < ns && j < nN) {
        const cpx<float> cv = cb[(long long)(kb + kk) * ns + n];
        v = (j & 1) ? cv.im : cv.re;
      }
      if (BF16)
        put_bf16(bhi, kmaj16(j, kk), v);
      else
        put_split(bhi, blo, kmaj(j, kk), v);
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma::fence_after_sync();
      if (BF16)
        issue_stage_bf16(tmem, umma::smem_addr(ahi), umma::smem_addr(bhi), idesc, step == 0);
      else
        issue_stage(tmem, umma::smem_addr(ahi), umma::smem_addr(alo), umma::smem_addr(bhi),
                    umma::smem_addr(blo), idesc, step == 0);
      umma::mma_commit(mb);
    }
    issued = step + 1;
  }
  if (issued > 0) {  // the last issued commit covers every MMA issued before it
    const bool done = umma::mbar_wait_bounded(mb, (issued - 1) & 1, kWaitLimit);
    ok = ok && done;
  }
  ok = __syncthreads_and(ok) != 0;
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  umma::fence_after_sync();
  const long long r = r0 + warp * 32 + lane;
  for (int j0 = 0; j0 < nN; j0 += 16) {
    float v[16];
    if (issued > 0 && ok) {
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int n = n0 + (j0 >> 1) + i;
      if (n < ns && r < nd) x0[((long long)b * ns + n) * nd + r] = mk<float>(v[2 * i], v[2 * i + 1]);
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 256);
}

// C_b = G_b / (eps_k - eps_n - i w_b) is formed by k_gram_coef (dense.cu).
template <typename T>
cudaError_t gram_coef(int ns, int nb, int nchunk, const double* gpart, const double* eps,
                      const double* omega, const int* active, double dV, cpx<T>* cmat,
                      cudaStream_t s);

template <bool BF16>
static cudaError_t tc_attr() {
  static bool attr = false;  // per process; the attribute is the same on every device
  if (attr) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (BF16 ? 4 : 8) * kTileBytes128);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_x0_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (BF16 ? 3 : 6) * kTileBytes128);
  if (e != cudaSuccess) return e;
  attr = true;
  return cudaSuccess;
}

cudaError_t galerkin_guess_tc(long long nd, int ns, int nb, const float* psi, const double* eps,
                              const double* omega, const float* u, const int* probe_active,
                              double dV, double* gpart, int nchunk, cpx<float>* cmat,
                              cpx<float>* x0, int* err, cudaStream_t s, bool bf16,
                              int test_expire) {
  cudaError_t e = bf16 ? tc_attr<true>() : tc_attr<false>();
  if (e != cudaSuccess) return e;
  const long long chunk_len = (nd + nchunk - 1) / nchunk;
  const int nt = (ns + 127) / 128;
  const int nN = std::min(128, ((ns + 15) / 16) * 16);
  dim3 g1(nt * nt, nb, nchunk);
  if (bf16)
    k_gram_tc<true><<<g1, 128, 4 * kTileBytes128, s>>>(nd, ns, psi, u, probe_active, nchunk,
                                                       chunk_len, nt, nN, gpart, err,
                                                       test_expire);
  else
    k_gram_tc<false><<<g1, 128, 8 * kTileBytes128, s>>>(nd, ns, psi, u, probe_active, nchunk,
                                                        chunk_len, nt, nN, gpart, err,
                                                       test_expire);
  e = gram_coef<float>(ns, nb, nchunk, gpart, eps, omega, probe_active, dV, cmat, s);
  if (e != cudaSuccess) return e;
  const int nN2 = std::min(256, ((2 * ns + 15) / 16) * 16);
  dim3 g3((unsigned)((nd + 127) / 128), nb * nt);
  if (bf16)
    k_x0_tc<true><<<g3, 128, 3 * kTileBytes128, s>>>(nd, ns, psi, cmat, probe_active, nt, nN2, x0,
                                                     err, test_expire);
  else
    k_x0_tc<false><<<g3, 128, 6 * kTileBytes128, s>>>(nd, ns, psi, cmat, probe_active, nt, nN2,
                                                      x0, err, test_expire);
  note_launch(3);
  return cudaGetLastError();
}

}  // namespace rpa
