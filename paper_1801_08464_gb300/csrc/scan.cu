// scan.cu -- device memory accounting, error words and exclusive scans.
#include "common.cuh"

namespace mgr {

std::atomic<unsigned long long> g_launch_count{0};
std::atomic<unsigned long long> g_wait_count{0};

void* dev_alloc(Ctx& c, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, c.s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(MGR_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  Ctx& a = c.acct ? *c.acct : c;
  std::unique_lock<std::mutex> lock;
  if (c.mu) lock = std::unique_lock<std::mutex>(*c.mu);
  a.bytes += (int64_t)bytes;
  if (a.bytes > a.peak) a.peak = a.bytes;
  return p;
}

void dev_free(Ctx& c, void* p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, c.s);
  Ctx& a = c.acct ? *c.acct : c;
  std::unique_lock<std::mutex> lock;
  if (c.mu) lock = std::unique_lock<std::mutex>(*c.mu);
  a.bytes -= (int64_t)bytes;
}

void check_errors(Ctx& c, const char* phase) {
  int e = read_scalar(c, c.d_err);
  if (!e) return;
  CU(cudaMemsetAsync(c.d_err, 0, sizeof(int), c.s));
  std::string w = std::string(phase) + ":";
  if (e & EBIT_PATTERN) throw Error(MGR_ERR_INVALID_ARG, w + " malformed matrix pattern or cf_marker");
  if (e & EBIT_CAPACITY) throw Error(MGR_ERR_UNSUPPORTED, w + " a row exceeds a kernel work limit");
  if (e & EBIT_SINGULAR) throw Error(MGR_ERR_SINGULAR, w + " zero or non-finite pivot");
  if (e & EBIT_NONFINITE) throw Error(MGR_ERR_BREAKDOWN, w + " non-finite value");
  throw Error(MGR_ERR_CUDA, w + " unknown device error bits");
}

// ---- three-phase exclusive scan: block sums, scan of the sums (recursive), block-local scan -----
constexpr int SCAN_T = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <class T>
__device__ T block_excl_scan(T v, T* sh, T* total) {
  // warp-level inclusive scan, then scan of the warp totals
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < SCAN_T / 32) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_T / 32) sh[lane] = w;
  }
  __syncthreads();
  T before = (wid > 0) ? sh[wid - 1] : T(0);
  if (total) *total = sh[SCAN_T / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <class TI, class TO>
__global__ void __launch_bounds__(SCAN_T) k_tile_sums(const TI* in, int64_t n, TO* sums) {
  __shared__ TO sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  TO s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + (int64_t)t * SCAN_T + threadIdx.x;
    if (i < n) s += (TO)in[i];
  }
  TO tot;
  block_excl_scan<TO>(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class TI, class TO>
__global__ void __launch_bounds__(SCAN_T) k_tile_scan(const TI* in, int64_t n, const TO* offs, TO* out, bool write_total) {
  __shared__ TO sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  TO v[SCAN_ITEMS];
  TO s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    v[t] = (i < n) ? (TO)in[i] : TO(0);
    s += v[t];
  }
  TO tot;
  TO pre = block_excl_scan<TO>(s, sh, &tot) + (offs ? offs[blockIdx.x] : TO(0));
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    if (i < n) out[i] = pre;
    pre += v[t];
  }
  if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_T - 1) out[n] = pre;
}

template <class TI, class TO>
static void scan_impl(Ctx& c, const TI* in, TO* out, int64_t n) {
  if (n <= 0) {
    CU(cudaMemsetAsync(out, 0, sizeof(TO), c.s));
    return;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_tile_scan<TI, TO><<<1, SCAN_T, 0, c.s>>>(in, n, nullptr, out, true);
    CU_LAUNCH();
    return;
  }
  DBuf<TO> sums(c, tiles), offs(c, tiles + 1);
  k_tile_sums<TI, TO><<<(unsigned)tiles, SCAN_T, 0, c.s>>>(in, n, sums.p);
  CU_LAUNCH();
  scan_impl<TO, TO>(c, sums.p, offs.p, tiles);
  k_tile_scan<TI, TO><<<(unsigned)tiles, SCAN_T, 0, c.s>>>(in, n, offs.p, out, false);
  CU_LAUNCH();
  // total: out[n] = offs[tiles]
  CU(cudaMemcpyAsync(out + n, offs.p + tiles, sizeof(TO), cudaMemcpyDeviceToDevice, c.s));
}

void scan_excl_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n) { scan_impl<int64_t, int64_t>(c, in, out, n); }
void scan_excl_i32(Ctx& c, const int32_t* in, int32_t* out, int64_t n) { scan_impl<int32_t, int32_t>(c, in, out, n); }

int64_t counts_to_rowptr(Ctx& c, const int64_t* counts, int64_t* rowptr, int64_t n) {
  scan_excl_i64(c, counts, rowptr, n);
  return read_scalar(c, rowptr + n);
}

template <class T>
__global__ void k_fill(T* p, T v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}
void fill_i64(Ctx& c, int64_t* p, int64_t v, int64_t n) {
  if (n <= 0) return;
  k_fill<<<grid_for(n, 256, 4096), 256, 0, c.s>>>(p, v, n);
  CU_LAUNCH();
}
void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n) {
  if (n <= 0) return;
  k_fill<<<grid_for(n, 256, 4096), 256, 0, c.s>>>(p, v, n);
  CU_LAUNCH();
}
void fill_f64(Ctx& c, double* p, double v, int64_t n) {
  if (n <= 0) return;
  k_fill<<<grid_for(n, 256, 4096), 256, 0, c.s>>>(p, v, n);
  CU_LAUNCH();
}

}  // namespace mgr
