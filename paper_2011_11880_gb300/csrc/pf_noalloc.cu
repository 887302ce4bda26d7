// Allocation-free F / J evaluation.
//
// Some callers cannot call cudaMalloc at the point where they evaluate: code
// that must not synchronise the device (cudaMalloc and cudaFree can
// serialise against running work), hosts that budget every byte of device
// memory up front, or plug-in layers that may only use memory handed to
// them.  pf_residual_jacobian_static serves them: it allocates nothing.
// Inputs, outputs and the built context come from the caller; the only
// scratch the evaluation needs -- the 32-byte per-bus record of every bus of
// every instance (the unit phasor (cos theta, sin theta) and V in fixed point,
// and 1/V) -- lives in g_static_phasor below, a fixed device array that
// exists on every GPU that loads this library until the process exits.  (A
// context tuned to form the records inside the fused kernel, fuse_phasor = 1,
// uses the array only for buses with more than 32 neighbours.)
#include <mutex>
#include <string>
#include <vector>

#include "pf_internal.cuh"

namespace pf {
namespace {

// Capacity of the static scratch: 2^18 instance-buses, one 32-byte record
// each: 8 MiB.
constexpr int64_t kStaticPhasorBuses = int64_t(1) << 18;

static __device__ __align__(256) double2 g_static_phasor[2 * kStaticPhasorBuses];

std::mutex g_setup_mutex;
std::vector<double2 *> g_setup_address;   // device address of g_static_phasor, per device

// Once per device, with that device current: look up the device address of
// the array.  In host code the name g_static_phasor is only a host-side
// stand-in; a kernel must be given this address instead.
int static_scratch(double2 **out) {
  int dev = 0;
  PF_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if ((int)g_setup_address.size() <= dev) g_setup_address.resize(dev + 1, nullptr);
  if (!g_setup_address[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_phasor);
    if (e != cudaSuccess)
      return fail(PF_ERR_CUDA, std::string("cudaGetSymbolAddress(g_static_phasor): ") + cudaGetErrorString(e));
    g_setup_address[dev] = static_cast<double2 *>(p);
  }
  *out = g_setup_address[dev];
  return PF_OK;
}

}  // namespace
}  // namespace pf

extern "C" int pf_residual_jacobian_static(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream) {
  pf::Ctx *c = pf::ctx_of(ctx);
  if (!c) return pf::fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(*c);
  if (!x) return pf::fail(PF_ERR_INVALID, "x is NULL");
  if (c->v.n_bus_inst > pf::kStaticPhasorBuses)
    return pf::fail(PF_ERR_UNSUPPORTED,
                    "pf_residual_jacobian_static: the context has " + std::to_string(c->v.n_bus_inst) +
                        " buses over all instances; the static scratch holds at most " +
                        std::to_string(pf::kStaticPhasorBuses) + " (use pf_residual_jacobian)");
  double2 *scratch = nullptr;
  PF_TRY(pf::static_scratch(&scratch));
  // Nothing in the array must start at zero: the phasor kernel rewrites every
  // entry the fused kernel then reads.
  return pf::launch_eval_scratch(*c, x, F, vals, scratch, static_cast<cudaStream_t>(stream));
}
