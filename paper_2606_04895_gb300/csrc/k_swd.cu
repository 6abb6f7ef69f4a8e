// k_swd.cu -- sliced Wasserstein distance (Sec. 4.1): projection directions, projections of the
// draws and of a reference set onto them, per-direction sorting, and the 1-D Wasserstein-1
// distance of each sorted pair.  Everything in FP64; the distance is a metric, not a step of
// the sampler.
#include <cub/device/device_segmented_radix_sort.cuh>

#include "launch.h"

namespace bst {

namespace {
inline int blocks_for(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

// first index of the sorted v[0..n) with v[i] >= x (lower) or v[i] > x (upper)
__device__ __forceinline__ long long bound_of(const double *v, long long n, double x, bool upper) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (upper ? (v[mid] <= x) : (v[mid] < x)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
}  // namespace

constexpr uint32_t kSwd = 9;  // Philox purpose of the directions (after the initial positions' 8)

// Direction k: the normals 0..d-1 of stream (k, 0, kSwd) divided by their Euclidean norm
// (uniform on the unit sphere); U[k][d].
__global__ void swd_directions_kernel(uint64_t seed, int n_proj, int d, double *U) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_proj) return;
  double u[kMaxD];
  draw_normals<double>(seed, static_cast<uint32_t>(k), 0u, kSwd, d, u);
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += u[i] * u[i];
  const double r = sqrt(s);
  for (int i = 0; i < d; ++i) U[static_cast<size_t>(k) * d + i] = u[i] / r;
}

// out[kk * ld + i] = x_i . u_kk for kk < nk and rows i < n_rows of X[n_rows][d]; one thread per
// row (the row in registers, the directions read through the cache), stores coalesced over i.
template <typename R>
__global__ void swd_project_kernel(const R *X, long long n_rows, int d, const double *U, int nk, double *out,
                                   long long ld) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  double x[kMaxD];
#pragma unroll
  for (int j = 0; j < kMaxD; ++j) x[j] = j < d ? static_cast<double>(X[i * d + j]) : 0.0;
  for (int kk = 0; kk < nk; ++kk) {
    const double *u = U + static_cast<size_t>(kk) * d;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kMaxD; ++j)
      if (j < d) s += x[j] * u[j];
    out[kk * ld + i] = s;
  }
}

// 1-D Wasserstein-1 distance of the sorted samples a[0..n) and b[0..m) (segment kk of `sorted`:
// a at kk (n + m), b right after it), as the integral of |F_a - F_b| over x.  In the merged
// order (a before b at equal values) each element owns the gap to its successor, on which
// F_a = ca / n and F_b = cb / m hold with ca, cb the counts of values <= the element (exact
// wherever the gap is not zero); the weight |ca m - cb n| / (n m) is formed in integers.  One
// block per direction, partial sums reduced in a fixed order.
constexpr int kSwdThreads = 256;
__global__ void __launch_bounds__(kSwdThreads) swd_w1_kernel(const double *sorted, long long n, long long m,
                                                            double *w1) {
  __shared__ double part[kSwdThreads];
  const double *a = sorted + static_cast<long long>(blockIdx.x) * (n + m), *b = a + n;
  const double inv_nm = 1.0 / (static_cast<double>(n) * static_cast<double>(m));
  double acc = 0.0;
  for (long long e = threadIdx.x; e < n + m; e += kSwdThreads) {
    double x, nxt = INFINITY;
    long long ca, cb;
    if (e < n) {
      x = a[e];
      if (e + 1 < n) nxt = a[e + 1];
      const long long lb = bound_of(b, m, x, false);
      if (lb < m) nxt = fmin(nxt, b[lb]);
      ca = e + 1;
      cb = bound_of(b, m, x, true);
    } else {
      const long long k = e - n;
      x = b[k];
      if (k + 1 < m) nxt = b[k + 1];
      const long long ub = bound_of(a, n, x, true);
      if (ub < n) nxt = fmin(nxt, a[ub]);
      ca = ub;
      cb = k + 1;
    }
    if (nxt > x && nxt < INFINITY) {
      const long long wgt = ca * m - cb * n;
      acc += (nxt - x) * (static_cast<double>(wgt < 0 ? -wgt : wgt) * inv_nm);
    }
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kSwdThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) w1[blockIdx.x] = part[0];
}

cudaError_t launch_swd_directions(uint64_t seed, int n_proj, int d, double *U, cudaStream_t s) {
  swd_directions_kernel<<<blocks_for(n_proj, 128), 128, 0, s>>>(seed, n_proj, d, U);
  return cudaGetLastError();
}
cudaError_t launch_swd_project_f32(const float *X, long long n_rows, int d, const double *U, int nk, double *out,
                                   long long ld, cudaStream_t s) {
  if (n_rows > 0) swd_project_kernel<float><<<blocks_for(n_rows, 128), 128, 0, s>>>(X, n_rows, d, U, nk, out, ld);
  return cudaGetLastError();
}
cudaError_t launch_swd_project_f64(const double *X, long long n_rows, int d, const double *U, int nk, double *out,
                                   long long ld, cudaStream_t s) {
  if (n_rows > 0) swd_project_kernel<double><<<blocks_for(n_rows, 128), 128, 0, s>>>(X, n_rows, d, U, nk, out, ld);
  return cudaGetLastError();
}
cudaError_t swd_sort_segments(void *temp, size_t &temp_bytes, const double *in, double *out, int n_items,
                              int n_segments, const int *offsets, cudaStream_t s) {
  return cub::DeviceSegmentedRadixSort::SortKeys(temp, temp_bytes, in, out, n_items, n_segments, offsets, offsets + 1,
                                                 0, 64, s);
}
cudaError_t launch_swd_w1(const double *sorted, long long n, long long m, int nk, double *w1, cudaStream_t s) {
  if (nk > 0) swd_w1_kernel<<<nk, kSwdThreads, 0, s>>>(sorted, n, m, w1);
  return cudaGetLastError();
}

}  // namespace bst
