// noalloc.cu -- block transpose of a 3x3 BSR matrix that allocates no memory.
//
// Same result as mgr_bsr3_transpose, but its working memory (per-column counters and the source
// block index of every transposed block) lives in one file-scope device array of fixed size instead
// of being allocated per call.  For callers that cannot allocate device memory at call time: code
// running under a caller-owned memory budget or pool that forbids hidden allocations, code whose
// latency cannot absorb an allocation, or a host application that hands this library only the
// buffers it owns.
#include <mutex>

#include "apply.cuh"

namespace mgr {
namespace {

constexpr int64_t NA_MAX_NB = 1 << 16;    // block rows
constexpr int64_t NA_MAX_NNZB = 1 << 19;  // stored blocks

// counters [NA_MAX_NB + 1], one error word, then source indices [NA_MAX_NNZB]; every GPU that
// loads the library holds this array (about 4.7 MB) until the process exits
constexpr int64_t NA_FLAG = NA_MAX_NB + 1;
constexpr int64_t NA_SRC = NA_MAX_NB + 2;
static __device__ __align__(256) unsigned long long g_transpose_scratch[NA_SRC + NA_MAX_NNZB];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per device.
void* scratch_address() {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) throw Error(MGR_ERR_UNSUPPORTED, "device index beyond 64");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    CU(cudaGetSymbolAddress(&p, g_transpose_scratch));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

__global__ void k_na_zero(int64_t n, unsigned long long* a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = 0;
}
// The input is checked before anything is written through it: the row pointers must run from 0 to
// nnzb without decreasing, and every column must lie in [0, nb).  A violation sets the error word
// and the later kernels write nothing, so a malformed matrix can never move a write outside the
// fixed array or the caller's output buffers.
__global__ void k_na_check_rows(int64_t nb, int64_t nnzb, const int64_t* rp, unsigned long long* flag) {
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nb; I += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = rp[I], b = rp[I + 1];
    bool bad = a < 0 || b < a || b > nnzb || (I == 0 && a != 0) || (I == nb - 1 && b != nnzb);
    if (bad) atomicOr(flag, 1ull);
  }
}
__global__ void k_na_count(int64_t nb, int64_t nnzb, const int32_t* ci, unsigned long long* cnt,
                           unsigned long long* flag) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t J = ci[k];
    if (J < 0 || J >= nb) {
      atomicOr(flag, 2ull);
      continue;
    }
    atomicAdd(&cnt[J], 1ull);
  }
}
// single-block exclusive scan of n <= NA_MAX_NB counts into rpt[0..n]
__global__ void __launch_bounds__(1024) k_na_scan(int64_t n, const unsigned long long* cnt, int64_t* rpt) {
  __shared__ int64_t wsum[32];
  int64_t per = (n + blockDim.x - 1) / blockDim.x;
  int64_t i0 = threadIdx.x * per;
  int64_t s = 0;
  for (int64_t t = 0; t < per && i0 + t < n; ++t) s += (int64_t)cnt[i0 + t];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t y = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    wsum[lane] = y;
  }
  __syncthreads();
  int64_t pre = (wid ? wsum[wid - 1] : 0) + x - s;
  for (int64_t t = 0; t < per && i0 + t < n; ++t) {
    rpt[i0 + t] = pre;
    pre += (int64_t)cnt[i0 + t];
  }
  if (threadIdx.x == blockDim.x - 1) rpt[n] = wsum[31];
}
__global__ void k_na_scatter(int64_t nb, const int64_t* rp, const int32_t* ci, const int64_t* rpt,
                             unsigned long long* slot, int32_t* cit, int64_t* src, const unsigned long long* flag) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb || *flag) return;
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
    int32_t J = ci[k];
    int64_t d = rpt[J] + (int64_t)atomicAdd(&slot[J], 1ull);
    cit[d] = (int32_t)I;
    src[d] = k;
  }
}
// order each transposed block row by column (insertion sort of short rows) and copy the blocks
// transposed
__global__ void k_na_sort_fill(int64_t nb, const int64_t* rpt, int32_t* cit, int64_t* src, const double* v, double* vt,
                               const unsigned long long* flag) {
  int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (J >= nb || *flag) return;
  int64_t b = rpt[J], e = rpt[J + 1];
  for (int64_t a = b + 1; a < e; ++a) {
    int32_t key = cit[a];
    int64_t s = src[a];
    int64_t t = a - 1;
    while (t >= b && cit[t] > key) { cit[t + 1] = cit[t]; src[t + 1] = src[t]; --t; }
    cit[t + 1] = key;
    src[t + 1] = s;
  }
  for (int64_t d = b; d < e; ++d) {
    const double* in = v + 9 * src[d];
    double* o = vt + 9 * d;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) o[3 * p + q] = in[3 * q + p];
  }
}

}  // namespace
}  // namespace mgr

using namespace mgr;

extern "C" mgr_status_t mgr_bsr3_transpose_noalloc(const mgr_bsr3_t* A, int64_t* rowptr_t, int32_t* colind_t,
                                                   double* values_t, void* cuda_stream) {
  if (!A || !rowptr_t || !colind_t || !values_t || A->nb <= 0 || A->nnzb < 0 || !A->rowptr || !A->colind ||
      !A->values)
    return MGR_ERR_INVALID_ARG;
  if (A->nb > NA_MAX_NB || A->nnzb > NA_MAX_NNZB) {
    fprintf(stderr, "[mgr] mgr_bsr3_transpose_noalloc: nb %lld > %lld or nnzb %lld > %lld\n", (long long)A->nb,
            (long long)NA_MAX_NB, (long long)A->nnzb, (long long)NA_MAX_NNZB);
    return MGR_ERR_UNSUPPORTED;
  }
  try {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long* cnt = static_cast<unsigned long long*>(scratch_address());
    unsigned long long* flag = cnt + NA_FLAG;
    int64_t* src = reinterpret_cast<int64_t*>(cnt + NA_SRC);
    int64_t nb = A->nb, nnzb = A->nnzb;
    k_na_zero<<<grid_for(nb + 1, 256, 1024), 256, 0, s>>>(nb + 1, cnt);
    CU_LAUNCH();
    k_na_zero<<<1, 32, 0, s>>>(1, flag);
    CU_LAUNCH();
    k_na_check_rows<<<grid_for(nb, 256, 1024), 256, 0, s>>>(nb, nnzb, A->rowptr, flag);
    CU_LAUNCH();
    if (nnzb > 0) {
      k_na_count<<<grid_for(nnzb, 256, 4096), 256, 0, s>>>(nb, nnzb, A->colind, cnt, flag);
      CU_LAUNCH();
    }
    k_na_scan<<<1, 1024, 0, s>>>(nb, cnt, rowptr_t);
    CU_LAUNCH();
    k_na_zero<<<grid_for(nb + 1, 256, 1024), 256, 0, s>>>(nb + 1, cnt);
    CU_LAUNCH();
    k_na_scatter<<<grid_for(nb, 256), 256, 0, s>>>(nb, A->rowptr, A->colind, rowptr_t, cnt, colind_t, src, flag);
    CU_LAUNCH();
    k_na_sort_fill<<<grid_for(nb, 256), 256, 0, s>>>(nb, rowptr_t, colind_t, src, A->values, values_t, flag);
    CU_LAUNCH();
    // read the error word back (a device-to-host copy into a host variable; no allocation)
    unsigned long long h_flag = 0;
    CU(cudaMemcpyAsync(&h_flag, flag, sizeof(h_flag), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h_flag) {
      fprintf(stderr, "[mgr] mgr_bsr3_transpose_noalloc: malformed input (%s%s)\n",
              (h_flag & 1ull) ? "row pointers not 0..nnzb non-decreasing" : "",
              (h_flag & 2ull) ? ((h_flag & 1ull) ? ", column outside [0, nb)" : "column outside [0, nb)") : "");
      return MGR_ERR_INVALID_ARG;
    }
    return MGR_OK;
  } catch (const Error& e) {
    fprintf(stderr, "[mgr] %s\n", e.what());
    return e.status;
  }
}
