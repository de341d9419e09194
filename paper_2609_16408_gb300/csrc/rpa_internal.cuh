// Internal declarations of the GB300 RPA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rpa.h"

namespace rpa {

// ---------------------------------------------------------------------------------------
// complex arithmetic (interleaved re/im, same layout as the ABI's complex arrays)
// ---------------------------------------------------------------------------------------
template <typename T>
struct __align__(sizeof(T) * 2) cpx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) {
  cpx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return mk(a.re * s, a.im * s); }
// a + s*b with s real
template <typename T>
__host__ __device__ __forceinline__ cpx<T> caxpy_r(cpx<T> a, T s, cpx<T> b) {
  return mk(a.re + s * b.re, a.im + s * b.im);
}

// ---------------------------------------------------------------------------------------
// operator descriptions passed to kernels by value
// ---------------------------------------------------------------------------------------
constexpr int kMaxRadius = 8;
constexpr int kProjChunk = 4;   // projectors per internal group (shared support)
constexpr int kMaxLanczos = 256;

template <typename T>
struct Stencil {
  int nx, ny, nz, R;
  int bcx, bcy, bcz;
  T cx[kMaxRadius + 1], cy[kMaxRadius + 1], cz[kMaxRadius + 1];  // -1/2 c_m / h^2, m >= 1
  T c0;                                                          // -1/2 c_0 sum 1/h^2
};

// Nonlocal projectors on the device, both orderings of the same entries.
template <typename T>
struct NonlocalDev {
  int ngroup;            // internal groups (<= kProjChunk projectors each)
  const int* g_off;      // ngroup + 1, group-major entry offsets
  const int* g_idx;      // grid index per group-major entry
  const T* g_chi;        // 4 values per group-major entry
  const T* coef;         // ngroup x 4: gamma * dV (0 for padding)
  const int* p_off;      // N_d + 1, point-major entry offsets
  const int* p_grp;      // group per point-major entry
  const T* p_chi;        // 4 values per point-major entry
  // overlaps of the projectors of groups with common support, S[g, h](l, m) = sum over the
  // common points of chi_{g,l} chi_{h,m}: for group g the groups s_nbr[s_off[g] ..
  // s_off[g + 1]) (g itself included) with one 4 x 4 block each (row-major) in s_blk
  const int* s_off;
  const int* s_nbr;
  const T* s_blk;
};

// ---------------------------------------------------------------------------------------
// device buffer helper
// ---------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf();
  cudaError_t ensure(size_t nbytes);  // grows (contents not kept)
  void release();
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// process-wide count of kernel launches issued by this library
void note_launch(int n = 1);

}  // namespace rpa

namespace rpa {

// error helpers (implemented in api.cu)
rpa_status fail(rpa_ctx* c, rpa_status st, const std::string& msg);
rpa_status cuda_fail(rpa_ctx* c, cudaError_t e, const char* where);

}  // namespace rpa
