// Deterministic integer primitives for the pattern builder.
#include "pf_sort_scan.cuh"
#include "pf_internal.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// exclusive prefix sum (block scan by warp shuffles + recursive block sums)
// ---------------------------------------------------------------------------

constexpr int kScanBlock = 1024;

template <class T>
__global__ void scan_blocks_kernel(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                                   int64_t *__restrict__ block_sums) {
  __shared__ int64_t warp_tot[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int64_t v = (i < n) ? (int64_t)in[i] : 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  const int64_t pre = (wid > 0 ? warp_tot[wid - 1] : 0) + x - v;
  if (i < n) out[i] = pre;
  if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = pre + v;
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void scan_total_kernel(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ total) {
  out[n] = (n > 0) ? *total : 0;
}

size_t scan_tmp_elems(int64_t n) {
  int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb <= 1) return 1;
  return (size_t)nb + (size_t)(nb + 1) + scan_tmp_elems(nb);
}

template <class T>
int exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  if (n <= 0) {
    PF_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return PF_OK;
  }
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  int64_t *sums = tmp;
  scan_blocks_kernel<T><<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, sums);
  PF_CUDA_TRY(cudaGetLastError());
  if (nb == 1) {
    scan_total_kernel<<<1, 1, 0, s>>>(out, n, sums);
    PF_CUDA_TRY(cudaGetLastError());
    return PF_OK;
  }
  int64_t *offs = tmp + nb;
  int rc = exclusive_scan<int64_t>(sums, offs, nb, tmp + nb + nb + 1, s);
  if (rc) return rc;
  scan_add_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(out, n, offs);
  scan_total_kernel<<<1, 1, 0, s>>>(out, n, offs + nb);
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

template int exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template int exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template int exclusive_scan<uint8_t>(const uint8_t *, int64_t *, int64_t, int64_t *, cudaStream_t);

// ---------------------------------------------------------------------------
// bitonic sort of (key, value) pairs, ascending by (key, value)
// ---------------------------------------------------------------------------

constexpr int kSortLocal = 2048;   // elements sorted per CTA in shared memory

__device__ __forceinline__ bool pair_greater(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
  return ka > kb || (ka == kb && va > vb);
}

__global__ void sort_pad_kernel(uint64_t *k, uint32_t *v, int64_t n, int64_t n_pad) {
  const int64_t i = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pad) {
    k[i] = ~0ull;
    v[i] = ~0u;
  }
}

// Runs stages k = k_lo .. k_hi (k_lo > 1 only when merging) restricted to
// j < L inside one CTA's chunk of L elements.
__global__ void bitonic_local_kernel(uint64_t *__restrict__ K, uint32_t *__restrict__ V, int L,
                                     int64_t k_lo, int64_t k_hi) {
  extern __shared__ unsigned char smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + L);
  const int64_t base = (int64_t)blockIdx.x * L;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    sk[t] = K[base + t];
    sv[t] = V[base + t];
  }
  for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
    int64_t j0 = (k <= L) ? (k >> 1) : (L >> 1);
    for (int64_t j = j0; j > 0; j >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (L >> 1); t += blockDim.x) {
        const int i = (int)(2 * j * (t / j) + (t % j));
        const int p = i + (int)j;
        const bool asc = (((base + i) & k) == 0);
        const uint64_t ka = sk[i], kb = sk[p];
        const uint32_t va = sv[i], vb = sv[p];
        if (pair_greater(ka, va, kb, vb) == asc) {
          sk[i] = kb; sk[p] = ka;
          sv[i] = vb; sv[p] = va;
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    K[base + t] = sk[t];
    V[base + t] = sv[t];
  }
}

__global__ void bitonic_global_kernel(uint64_t *__restrict__ K, uint32_t *__restrict__ V, int64_t n,
                                      int64_t k, int64_t j) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (n >> 1)) return;
  const int64_t i = 2 * j * (t / j) + (t % j);
  const int64_t p = i + j;
  const bool asc = ((i & k) == 0);
  const uint64_t ka = K[i], kb = K[p];
  const uint32_t va = V[i], vb = V[p];
  if (pair_greater(ka, va, kb, vb) == asc) {
    K[i] = kb; K[p] = ka;
    V[i] = vb; V[p] = va;
  }
}

int64_t sort_padded(int64_t n) {
  int64_t p = 2;
  while (p < n) p <<= 1;
  return p;
}

int bitonic_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, cudaStream_t s) {
  const int64_t np = sort_padded(n);
  if (np > n) {
    sort_pad_kernel<<<(unsigned)((np - n + 255) / 256), 256, 0, s>>>(keys, vals, n, np);
    PF_CUDA_TRY(cudaGetLastError());
  }
  const int L = (int)(np < kSortLocal ? np : kSortLocal);
  const int threads = L / 2 < 1024 ? L / 2 : 1024;
  const size_t smem = (size_t)L * (sizeof(uint64_t) + sizeof(uint32_t));
  const unsigned nblk = (unsigned)(np / L);
  bitonic_local_kernel<<<nblk, threads, smem, s>>>(keys, vals, L, 2, L);
  PF_CUDA_TRY(cudaGetLastError());
  for (int64_t k = 2 * (int64_t)L; k <= np; k <<= 1) {
    for (int64_t j = k >> 1; j >= L; j >>= 1) {
      bitonic_global_kernel<<<(unsigned)((np / 2 + 255) / 256), 256, 0, s>>>(keys, vals, np, k, j);
    }
    bitonic_local_kernel<<<nblk, threads, smem, s>>>(keys, vals, L, k, k);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

}  // namespace pf
