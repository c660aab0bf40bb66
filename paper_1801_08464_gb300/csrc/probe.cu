// probe.cu -- FP64 FMA-rate probe: the denominator of the roofline of the FP64-bound Krylov kernels.
//
// GB300 issues few FP64 FMAs per clock (the Krylov SpMV and the Gram-Schmidt kernels reach its rate
// before HBM bandwidth), so their roofline is this measured rate, not a nominal figure.  The kernel
// is eight independent FMA chains per thread over a full-occupancy grid: the latency of each chain
// is hidden by the other chains and warps, and nothing but the FMAs and a counted loop is issued.
// Every operand is a register (the multiplier and addend are loaded from device memory at entry):
// an FMA that takes an operand from the constant bank issues at about 0.84 of the register rate on
// this GPU (measured), and the solver's FMAs take theirs from registers.
#include "common.cuh"

namespace mgr {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_fma_chains(int64_t len, const double* ab, double sentinel,
                                                                   double* out) {
  const double a = ab[0], b = ab[1];
  double x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int64_t k = 0; k < len; k += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == sentinel) out[0] = s;  // never true for the arguments used; keeps the chains live
}

}  // namespace
}  // namespace mgr

using namespace mgr;

extern "C" mgr_status_t mgr_probe_fp64_fma(int64_t chain_len, int launches, void* cuda_stream, double* gfma_per_s,
                                           double* ms_per_launch) {
  if (chain_len <= 0 || (chain_len & 3) || launches <= 0 || !gfma_per_s) return MGR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mgr_status_t st = MGR_OK;
  try {
    int dev = 0, sms = 0, per_sm = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma_chains, PROBE_THREADS, 0));
    unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    CU(cudaMalloc(&out, 3 * sizeof(double)));  // multiplier, addend, sink
    const double ab[2] = {0.999999, 1e-6};
    CU(cudaMemcpyAsync(out, ab, sizeof(ab), cudaMemcpyHostToDevice, s));
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    k_fp64_fma_chains<<<grid, PROBE_THREADS, 0, s>>>(chain_len, out, -1.0, out + 2);  // warm-up
    CU_LAUNCH();
    CU(cudaEventRecord(e0, s));
    for (int i = 0; i < launches; ++i) {
      k_fp64_fma_chains<<<grid, PROBE_THREADS, 0, s>>>(chain_len, out, -1.0, out + 2);
      CU_LAUNCH();
    }
    CU(cudaEventRecord(e1, s));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    double fmas = (double)grid * PROBE_THREADS * PROBE_CHAINS * (double)chain_len * launches;
    *gfma_per_s = fmas / (ms * 1e-3) / 1e9;
    if (ms_per_launch) *ms_per_launch = ms / launches;
  } catch (const Error& e) {
    fprintf(stderr, "[mgr] %s\n", e.what());
    st = e.status;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return st;
}
