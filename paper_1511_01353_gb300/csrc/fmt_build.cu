// fmt_build.cu -- oct_build kernels: input check and max|f| (tau), Morton
// codes, stable LSD radix sort of the codes, gather into sorted SoA.
//
// Sorting once by Morton code replaces the per-node FMT_Ordered_by_Octant of
// Alg. 1: after the sort every octree node at every depth is a contiguous
// range of the sorted arrays, so the children of a node are found by binary
// search instead of by moving points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fmt_internal.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per tile

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// problem of point i (problems are contiguous ranges of the input)
__device__ __forceinline__ int problem_of_point(const fmt_problem* __restrict__ prob, int P, int64_t i) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prob[mid].start <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per-problem max |f| and a finiteness check of every coordinate and value.
// A block whose points all belong to one problem reduces in shared memory and
// issues one atomic; otherwise every thread updates its problem directly.
__global__ void __launch_bounds__(256) k_check_maxabs(int64_t n, const double* __restrict__ x,
                                                      const double* __restrict__ y,
                                                      const double* __restrict__ z,
                                                      const double* __restrict__ f,
                                                      const fmt_problem* __restrict__ prob, int P,
                                                      unsigned long long* maxbits, int* err) {
  __shared__ double red[8];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rounds = (n + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t base = r * stride + (int64_t)blockIdx.x * blockDim.x;
    const int64_t i = first + r * stride;
    const int64_t last = (base + blockDim.x < n ? base + blockDim.x : n) - 1;
    const int p0 = base < n ? problem_of_point(prob, P, base) : 0;
    const int p1 = base < n ? problem_of_point(prob, P, last) : 0;
    double m = 0.0;
    bool bad = false;
    if (i < n) {
      const double a = x[i], b = y[i], c = z[i], v = f[i];
      bad = !isfinite(a) || !isfinite(b) || !isfinite(c) || !isfinite(v);
      m = fabs(v);
      if (p0 != p1 && isfinite(m) && m > 0.0)
        atomicMax(&maxbits[problem_of_point(prob, P, i)], (unsigned long long)__double_as_longlong(m));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, FMT_ERR_NONFINITE);
    if (p0 == p1) {  // block-uniform
      m = warp_max(m);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
      __syncthreads();
      if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_max(v);
        // non-negative doubles order like their bit patterns
        if (threadIdx.x == 0 && isfinite(v) && v > 0.0)
          atomicMax(&maxbits[p0], (unsigned long long)__double_as_longlong(v));
      }
      __syncthreads();
    }
  }
}

// Sort key: problem id above the top sort_bits bits of the Morton code.
template <typename K>
__global__ void __launch_bounds__(256) k_morton(int64_t n, const double* __restrict__ x,
                                                const double* __restrict__ y,
                                                const double* __restrict__ z,
                                                const fmt_problem* __restrict__ prob, int P, int sort_shift,
                                                int sort_bits, K* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = P > 1 ? problem_of_point(prob, P, i) : 0;
    if (!FMT_CHECK(fmt_in(p, P), CK_BUILD_INDEX)) continue;
    const fmt_problem& pr = prob[p];
    const uint64_t code = fmt_spread3(fmt_quant(x[i], pr.lo[0], pr.S)) |
                          (fmt_spread3(fmt_quant(y[i], pr.lo[1], pr.S)) << 1) |
                          (fmt_spread3(fmt_quant(z[i], pr.lo[2], pr.S)) << 2);
    keys[i] = (K)(((uint64_t)p << sort_bits) | (code >> sort_shift));
    vals[i] = (uint32_t)i;
  }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                             uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// block-wide exclusive scan of one value per thread (256 threads)
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[8];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  uint32_t wbase = 0, tot = 0;
  for (int w = 0; w < 8; ++w) {
    uint32_t c = ws[w];
    if (w < warp) wbase += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return wbase + inc - v;
}

// per digit: exclusive scan over tiles (in place); digit totals out
__global__ void __launch_bounds__(256) k_radix_scan_tiles(uint32_t* __restrict__ hist, int ntiles,
                                                          uint32_t* __restrict__ bintotal) {
  uint32_t* row = hist + (int64_t)blockIdx.x * ntiles;
  uint32_t carry = 0;
  for (int t0 = 0; t0 < ntiles; t0 += 256) {
    int t = t0 + threadIdx.x;
    uint32_t v = t < ntiles ? row[t] : 0u;
    uint32_t tot;
    uint32_t ex = block_exscan256(v, &tot);
    if (t < ntiles) row[t] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bintotal[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(256) k_radix_scan_bins(uint32_t* __restrict__ bintotal) {
  uint32_t tot;
  uint32_t v = bintotal[threadIdx.x];
  uint32_t ex = block_exscan256(v, &tot);
  bintotal[threadIdx.x] = ex;
}

// Stable scatter: inside a tile, keys keep their order (round, warp, lane).
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K* __restrict__ keys,
                                                                const uint32_t* __restrict__ vals, int64_t n,
                                                                int shift, const uint32_t* __restrict__ hist,
                                                                const uint32_t* __restrict__ binbase, int ntiles,
                                                                K* __restrict__ okeys, uint32_t* __restrict__ ovals) {
  __shared__ uint32_t cnt[8][256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t gofs[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  run[tid] = 0;
  gofs[tid] = binbase[tid] + hist[(int64_t)tid * ntiles + blockIdx.x];
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + tid;
    bool valid = i < n;
    K key = valid ? keys[i] : (K)0;
    uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
    for (int e = tid; e < 8 * 256; e += kSortThreads) (&cnt[0][0])[e] = 0u;
    __syncthreads();
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == (uint32_t)__popc(peers) - 1u) cnt[warp][d] = (uint32_t)__popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[tid];
      for (int w = 0; w < 8; ++w) {
        uint32_t c = cnt[w][tid];
        cnt[w][tid] = acc;
        acc += c;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid && FMT_CHECK((int64_t)gofs[d] + cnt[warp][d] + rank < n, CK_BUILD_INDEX)) {
      uint32_t pos = gofs[d] + cnt[warp][d] + rank;
      okeys[pos] = key;
      ovals[pos] = vals[i];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_gather(int64_t n, const uint32_t* __restrict__ perm,
                                                const double* __restrict__ x, const double* __restrict__ y,
                                                const double* __restrict__ z, const double* __restrict__ f,
                                                const fmt_problem* __restrict__ prob, int P,
                                                double* __restrict__ xs, double* __restrict__ ys,
                                                double* __restrict__ zs, double* __restrict__ rs,
                                                uint64_t* __restrict__ code) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = perm[i];
    const int p = P > 1 ? problem_of_point(prob, P, i) : 0;
    if (!FMT_CHECK((int64_t)j < n && fmt_in(p, P), CK_BUILD_INDEX)) continue;
    const double a = x[j], b = y[j], c = z[j];
    const fmt_problem& pr = prob[p];
    xs[i] = a;
    ys[i] = b;
    zs[i] = c;
    rs[i] = f[j];
    code[i] = fmt_spread3(fmt_quant(a, pr.lo[0], pr.S)) | (fmt_spread3(fmt_quant(b, pr.lo[1], pr.S)) << 1) |
              (fmt_spread3(fmt_quant(c, pr.lo[2], pr.S)) << 2);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = 152 * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_check_maxabs(int64_t n, const double* x, const double* y, const double* z,
                                const double* f, const fmt_problem* prob, int P, unsigned long long* d_maxbits,
                                int* d_err, cudaStream_t s) {
  k_check_maxabs<<<grid_for(n, 256), 256, 0, s>>>(n, x, y, z, f, prob, P, d_maxbits, d_err);
  return cudaGetLastError();
}

cudaError_t launch_morton(int64_t n, const double* x, const double* y, const double* z, const fmt_problem* prob,
                          int P, int sort_shift, int sort_bits, bool key64, void* keys, uint32_t* vals,
                          cudaStream_t s) {
  if (key64)
    k_morton<uint64_t><<<grid_for(n, 256), 256, 0, s>>>(n, x, y, z, prob, P, sort_shift, sort_bits,
                                                        (uint64_t*)keys, vals);
  else
    k_morton<uint32_t><<<grid_for(n, 256), 256, 0, s>>>(n, x, y, z, prob, P, sort_shift, sort_bits,
                                                        (uint32_t*)keys, vals);
  return cudaGetLastError();
}

size_t radix_sort_temp_bytes(int64_t n, bool /*key64*/) {
  int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  return (size_t)(256 * ntiles + 256) * sizeof(uint32_t);
}

template <typename K>
static cudaError_t radix_sort_impl(int64_t n, int bits, K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt,
                                   void* temp, K** keys_out, uint32_t** vals_out, cudaStream_t s) {
  int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  uint32_t* hist = (uint32_t*)temp;
  uint32_t* bintotal = hist + (int64_t)256 * ntiles;
  K *src = keys, *dst = keys_alt;
  uint32_t *vsrc = vals, *vdst = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<K><<<ntiles, kSortThreads, 0, s>>>(src, n, shift, hist, ntiles);
    k_radix_scan_tiles<<<256, 256, 0, s>>>(hist, ntiles, bintotal);
    k_radix_scan_bins<<<1, 256, 0, s>>>(bintotal);
    k_radix_scatter<K><<<ntiles, kSortThreads, 0, s>>>(src, vsrc, n, shift, hist, bintotal, ntiles, dst, vdst);
    K* tk = src;
    src = dst;
    dst = tk;
    uint32_t* tv = vsrc;
    vsrc = vdst;
    vdst = tv;
  }
  *keys_out = src;
  *vals_out = vsrc;
  return cudaGetLastError();
}

cudaError_t launch_radix_sort(int64_t n, int bits, bool key64, void* keys, uint32_t* vals, void* keys_alt,
                              uint32_t* vals_alt, void* temp, void** keys_out, uint32_t** vals_out,
                              cudaStream_t s) {
  if (n <= 0 || bits <= 0) {
    *keys_out = keys;
    *vals_out = vals;
    return cudaSuccess;
  }
  if (key64) {
    uint64_t* ko = nullptr;
    cudaError_t e = radix_sort_impl<uint64_t>(n, bits, (uint64_t*)keys, vals, (uint64_t*)keys_alt, vals_alt, temp,
                                              &ko, vals_out, s);
    *keys_out = ko;
    return e;
  }
  uint32_t* ko = nullptr;
  cudaError_t e = radix_sort_impl<uint32_t>(n, bits, (uint32_t*)keys, vals, (uint32_t*)keys_alt, vals_alt, temp,
                                            &ko, vals_out, s);
  *keys_out = ko;
  return e;
}

cudaError_t launch_gather(int64_t n, const uint32_t* perm, const double* x, const double* y,
                          const double* z, const double* f, const fmt_problem* prob, int P, double* xs, double* ys,
                          double* zs, double* rs, uint64_t* code, cudaStream_t s) {
  k_gather<<<grid_for(n, 256), 256, 0, s>>>(n, perm, x, y, z, f, prob, P, xs, ys, zs, rs, code);
  return cudaGetLastError();
}

#ifdef FMT_CHECKED
FMT_CHECK_READER(check_site_build)
#endif
