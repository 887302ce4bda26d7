// Measurement helper: the FP64 fused multiply-add rate this GPU sustains,
// the denominator of the FP64 fractions reported beside the evaluation's
// roofline.  Eight independent FMA chains per thread, 2,048 threads per SM
// (enough independent work to keep the FP64 pipe busy), timed with CUDA
// events on the caller's stream.
#include <string>

#include "pf_internal.cuh"

namespace pf {
namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

__global__ void __launch_bounds__(kPeakThreads) k_fp64_peak(int iters, double seed, double *out) {
  double a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + (double)(threadIdx.x + c) * 1e-9;
  const double b = 0.9999999, d = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) a[c] = __fma_rn(a[c], b, d);
  }
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) r += a[c];
  // one write per block keeps the chains live without touching memory per thread
  if (r == 12345.0) out[blockIdx.x] = r;
}

}  // namespace
}  // namespace pf

extern "C" int pf_fp64_peak(int32_t device, double *gops, double *ms, void *stream) {
  if (!gops) return pf::fail(PF_ERR_INVALID, "gops is NULL");
  const pf::DeviceGuard guard(device);
  if (guard.status) return pf::fail(PF_ERR_CUDA, "cannot make the device current");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  PF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = sms * pf::kPeakBlocksPerSm;
  double *out = nullptr;
  PF_CUDA_TRY(cudaMalloc(&out, sizeof(double) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PF_OK;
  float best = 0.0f;
  const int iters = 2048;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = pf::fail(PF_ERR_CUDA, "cudaEventCreate failed");
  } else {
    pf::k_fp64_peak<<<blocks, pf::kPeakThreads, 0, s>>>(16, 1.0, out);     // warm-up
    for (int rep = 0; rep < 3 && rc == PF_OK; ++rep) {
      cudaEventRecord(e0, s);
      pf::k_fp64_peak<<<blocks, pf::kPeakThreads, 0, s>>>(iters, 1.0 + rep, out);
      cudaEventRecord(e1, s);
      const cudaError_t err = cudaEventSynchronize(e1);
      if (err != cudaSuccess) {
        rc = pf::fail(PF_ERR_CUDA, std::string("FP64 peak kernel: ") + cudaGetErrorString(err));
        break;
      }
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep == 0 || t < best) best = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return rc;
  const double ops = (double)blocks * pf::kPeakThreads * iters * pf::kPeakChains;
  *gops = ops / (best * 1e-3) / 1e9;
  if (ms) *ms = best;
  return PF_OK;
}
