// Allocation-free dense inertia: the Bunch-Kaufman front elimination applied to one small dense
// pencil, with its working copy of a - sigma*b in a fixed file-scope device array instead of
// memory from cudaMalloc.
//
// Who needs it: code that must not allocate device memory at the point of the call, for example
// a caller running under a framework that owns all device memory through its own pool, or an
// embedded/real-time host loop where cudaMalloc's implicit synchronisation and possible failure
// are not acceptable.  Such a caller passes device pointers it already has (the matrices) and a
// host array for the result; this call touches no allocator.
//
// The array below is reserved on every GPU that loads the library, for the life of the process.
// Every call shares it, so calls that overlap on the GPU (several host threads, or several
// streams) race; callers must serialise them.  The counters are zeroed by the kernel at the start
// of every call; the matrix copy is fully overwritten before it is read.
#include <cstdint>
#include <mutex>

#include "kep_internal.h"

namespace kep {
namespace {

constexpr int kNoallocMaxN = 512;                       // largest supported order
constexpr int kNoallocThreads = 1024;

__device__ __align__(256) double g_noalloc_matrix[kNoallocMaxN * kNoallocMaxN];   // 2 MiB
__device__ __align__(256) long long g_noalloc_counts[4];

// Device addresses of the two arrays, looked up once per device (host code may not use the
// symbols' host-side names as device addresses).
constexpr int kMaxDevices = 64;
double* g_matrix_addr[kMaxDevices] = {};
long long* g_counts_addr[kMaxDevices] = {};

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = -1.0;
  for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) r = fmax(r, red[w]);
  return r;
}

// Full symmetric copy M = a - sigma*b (lower triangles of a and b read), then Bunch-Kaufman
// elimination over all n columns (alpha = (1+sqrt 17)/8), counting the signs of D's 1x1 and 2x2
// blocks.  Only the trailing matrix is updated: the inertia needs D, not L.
__global__ void __launch_bounds__(kNoallocThreads) dense_bk_inertia_kernel(
    int32_t n, const double* __restrict__ a, const double* __restrict__ b, int64_t lda,
    double sigma, double* M, long long* cnt) {
  __shared__ double red[kNoallocThreads / 32];
  __shared__ int32_t s_r, s_kind, s_piv;
  const int tid = threadIdx.x;
  if (tid < 4) cnt[tid] = 0;
  for (int64_t e = tid; e < static_cast<int64_t>(n) * n; e += blockDim.x) {
    const int32_t i = static_cast<int32_t>(e % n), j = static_cast<int32_t>(e / n);
    const int32_t lo = i > j ? i : j, hi = i > j ? j : i;
    M[e] = a[lo + hi * lda] - sigma * b[lo + hi * lda];
  }
  __syncthreads();
  const double alpha = kBKAlpha;
  int32_t k = 0;
  while (k < n) {
    // largest entry below the diagonal in column k and its row
    double v = -1.0;
    int32_t arg = -1;
    for (int32_t i = k + 1 + tid; i < n; i += blockDim.x) {
      const double x = fabs(M[i + static_cast<int64_t>(k) * n]);
      if (x > v) { v = x; arg = i; }
    }
    const double lam = fmax(block_max(v, red), 0.0);
    if (tid == 0) s_r = n;
    __syncthreads();
    if (arg >= 0 && v == lam && lam > 0.0) atomicMin(&s_r, arg);
    __syncthreads();
    const int32_t r = s_r;
    const double akk = fabs(M[k + static_cast<int64_t>(k) * n]);
    if (lam == 0.0 || akk >= alpha * lam) {
      if (tid == 0) { s_kind = 1; s_piv = k; }
    } else {
      double vr = -1.0;
      for (int32_t i = k + tid; i < n; i += blockDim.x)
        if (i != r) vr = fmax(vr, fabs(M[i + static_cast<int64_t>(r) * n]));
      const double sig = fmax(block_max(vr, red), 0.0);
      if (tid == 0) {
        if (akk * sig >= alpha * lam * lam) { s_kind = 1; s_piv = k; }
        else if (fabs(M[r + static_cast<int64_t>(r) * n]) >= alpha * sig) { s_kind = 1; s_piv = r; }
        else { s_kind = 2; s_piv = r; }
      }
    }
    __syncthreads();
    const int32_t kind = s_kind, piv = s_piv;
    const int32_t dst = kind == 1 ? k : k + 1;
    if (piv != dst) {           // symmetric interchange: rows, then columns
      for (int32_t j = tid; j < n; j += blockDim.x) {
        double* x = M + dst + static_cast<int64_t>(j) * n;
        double* y = M + piv + static_cast<int64_t>(j) * n;
        const double t = *x; *x = *y; *y = t;
      }
      __syncthreads();
      for (int32_t i = tid; i < n; i += blockDim.x) {
        double* x = M + i + static_cast<int64_t>(dst) * n;
        double* y = M + i + static_cast<int64_t>(piv) * n;
        const double t = *x; *x = *y; *y = t;
      }
      __syncthreads();
    }
    const int32_t s = k + kind;          // first trailing index
    if (kind == 1) {
      const double d = M[k + static_cast<int64_t>(k) * n];
      if (tid == 0) {
        if (d < 0) cnt[0]++; else if (d > 0) cnt[2]++; else cnt[1]++;
      }
      if (d != 0.0) {
        const int64_t len = n - s;
        for (int64_t e = tid; e < len * len; e += blockDim.x) {
          const int32_t i = s + static_cast<int32_t>(e % len), j = s + static_cast<int32_t>(e / len);
          M[i + static_cast<int64_t>(j) * n] -=
              M[i + static_cast<int64_t>(k) * n] * M[k + static_cast<int64_t>(j) * n] / d;
        }
      }
    } else {
      const double a11 = M[k + static_cast<int64_t>(k) * n];
      const double a21 = M[k + 1 + static_cast<int64_t>(k) * n];
      const double a22 = M[k + 1 + static_cast<int64_t>(k + 1) * n];
      const double det = a11 * a22 - a21 * a21, tr = a11 + a22;
      if (tid == 0) {
        if (det < 0) { cnt[0]++; cnt[2]++; }
        else if (det > 0) { if (tr < 0) cnt[0] += 2; else cnt[2] += 2; }
        else if (tr < 0) { cnt[0]++; cnt[1]++; }
        else if (tr > 0) { cnt[2]++; cnt[1]++; }
        else cnt[1] += 2;
      }
      if (det != 0.0) {
        const int64_t len = n - s;
        for (int64_t e = tid; e < len * len; e += blockDim.x) {
          const int32_t i = s + static_cast<int32_t>(e % len), j = s + static_cast<int32_t>(e / len);
          const double wi0 = M[i + static_cast<int64_t>(k) * n], wi1 = M[i + static_cast<int64_t>(k + 1) * n];
          const double wj0 = M[k + static_cast<int64_t>(j) * n], wj1 = M[k + 1 + static_cast<int64_t>(j) * n];
          const double l0 = (a22 * wj0 - a21 * wj1) / det, l1 = (a11 * wj1 - a21 * wj0) / det;
          M[i + static_cast<int64_t>(j) * n] -= wi0 * l0 + wi1 * l1;
        }
      }
    }
    __syncthreads();
    k = s;
  }
}

std::mutex g_setup_mutex;   // host threads making their first call on a device at the same time

// Per-device lookup of the arrays' device addresses; the first call on a device does it.
kep_status noalloc_setup(int dev, double** m, long long** c) {
  if (dev < 0 || dev >= kMaxDevices) return KEP_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_matrix_addr[dev]) {
    void* pm = nullptr;
    void* pc = nullptr;
    if (cudaGetSymbolAddress(&pm, g_noalloc_matrix) != cudaSuccess) return KEP_ERR_CUDA;
    if (cudaGetSymbolAddress(&pc, g_noalloc_counts) != cudaSuccess) return KEP_ERR_CUDA;
    g_matrix_addr[dev] = static_cast<double*>(pm);
    g_counts_addr[dev] = static_cast<long long*>(pc);
  }
  *m = g_matrix_addr[dev];
  *c = g_counts_addr[dev];
  return KEP_OK;
}

}  // namespace
}  // namespace kep

extern "C" kep_status kep_dense_inertia_noalloc(int64_t n, const double* a, const double* b, int64_t lda,
                                                double sigma, void* stream, int64_t* out) {
  using namespace kep;
  if (n < 1 || n > kNoallocMaxN || lda < n || !a || !b || !out) return KEP_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KEP_ERR_CUDA;
  double* M = nullptr;
  long long* cnt = nullptr;
  kep_status st = noalloc_setup(dev, &M, &cnt);
  if (st != KEP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dense_bk_inertia_kernel<<<1, kNoallocThreads, 0, s>>>(static_cast<int32_t>(n), a, b, lda, sigma, M, cnt);
  if (cudaGetLastError() != cudaSuccess) return KEP_ERR_CUDA;
  long long h[4];
  if (cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return KEP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return KEP_ERR_CUDA;
  out[0] = h[0]; out[1] = h[1]; out[2] = h[2];
  return KEP_OK;
}
