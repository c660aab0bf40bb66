// common.cuh -- shared host/device utilities of the MGR-FGMRES library (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <initializer_list>
#include <map>
#include <mutex>
#include <set>
#include <stdexcept>
#include <vector>
#include <string>
#include <utility>

#include "mgr.h"

namespace mgr {

// ---------------------------------------------------------------------------------------------
// Errors: every failure becomes an Error carrying an mgr_status_t; the C-ABI layer converts it.
struct Error : std::runtime_error {
  mgr_status_t status;
  Error(mgr_status_t s, const std::string& what) : std::runtime_error(what), status(s) {}
};

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  mgr_status_t s = (e == cudaErrorMemoryAllocation) ? MGR_ERR_OOM : MGR_ERR_CUDA;
  throw Error(s, std::string(what) + ": " + cudaGetErrorString(e) + " at " + file + ":" + std::to_string(line));
}
#define CU(x) ::mgr::cuda_check((x), #x, __FILE__, __LINE__)
// Every kernel launch of the library is followed by CU_LAUNCH(), which checks it and counts it.
extern std::atomic<unsigned long long> g_launch_count;
// Every host wait on a stream (a scalar read-back, a synchronisation) is counted too: in the setup
// each one leaves the GPU idle while the host reads the value and issues the next launches.
extern std::atomic<unsigned long long> g_wait_count;
#define CU_LAUNCH()                                                                  \
  do {                                                                               \
    ::mgr::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__);      \
    ++::mgr::g_launch_count;                                                         \
  } while (0)

// Device error bits set by kernels (atomicOr) and checked by the host after a phase.
enum : int {
  EBIT_SINGULAR = 1,     // zero or non-finite pivot / diagonal
  EBIT_PATTERN = 2,      // malformed BSR pattern or marker
  EBIT_CAPACITY = 4,     // a per-row work bound exceeded a kernel limit
  EBIT_NONFINITE = 8,
};

// ---------------------------------------------------------------------------------------------
// Optional per-kernel timing: CUDA events recorded on the launching stream around each launch of a
// named kernel; elapsed times are summed when queried.
struct Prof {
  struct Rec {
    std::vector<cudaEvent_t> a, b;
    double ms = 0.0;
    int64_t n = 0;
    double bytes = 0.0;         // algorithmic bytes declared by the timed launches
    double bytes_stored = 0.0;  // bytes of the stored (compressed) operator forms the launches read
  };
  std::map<std::string, Rec> recs;
  std::set<std::string> only;  // when not empty, only these names are recorded
  std::vector<cudaEvent_t> pool;
  bool wants(const char* n) const { return only.empty() || only.count(n) != 0; }
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void settle() {  // fold recorded pairs into totals (synchronises on the events)
    for (auto& kv : recs) {
      Rec& r = kv.second;
      for (size_t i = 0; i < r.a.size(); ++i) {
        float t = 0.f;
        cudaEventSynchronize(r.b[i]);
        cudaEventElapsedTime(&t, r.a[i], r.b[i]);
        r.ms += t;
        r.n += 1;
        pool.push_back(r.a[i]);
        pool.push_back(r.b[i]);
      }
      r.a.clear();
      r.b.clear();
    }
  }
  ~Prof() {
    settle();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

constexpr int PIN_SLOTS = 16;

// Execution context: stream, device error word, allocation accounting.
struct Ctx {
  Prof* prof = nullptr;
  cudaStream_t s = nullptr;
  int* d_err = nullptr;        // device int, error bits
  void* h_pinned = nullptr;    // pinned host scratch of PIN_SLOTS 8-byte slots for read-backs (may be null)
  int64_t spgemm_stage = 0;    // staged products per SpGEMM batch (0: the library default)
  int64_t bytes = 0;           // bytes currently allocated through this context
  int64_t peak = 0;
  int num_sms = 152;
  bool pdl = true;             // programmatic dependent launch for the kernels launched with launch_pdl
  // a context on a second stream and host thread books its device bytes on `acct` (the handle's
  // main context), under `mu` while the two run at once
  Ctx* acct = nullptr;
  std::mutex* mu = nullptr;
};

struct ProfScope {
  Ctx& c;
  const char* name;
  cudaEvent_t e1 = nullptr;
  // bytes: the algorithmic bytes of the work inside the scope (each input element read once, each
  // output written once; a sparse entry counts its value and a 4-byte column index whatever form
  // the layout stores), summed per name for achieved-bandwidth figures.  stored: the same count
  // with the column indices as the layout stores them (one-byte codes, 16-bit offsets), when that
  // differs (negative: equal to bytes).
  bool on = false;
  ProfScope(Ctx& ctx, const char* n, double bytes = 0.0, double stored = -1.0) : c(ctx), name(n) {
    if (!n || !c.prof || !c.prof->wants(n)) return;
    on = true;
    cudaEvent_t e0 = c.prof->get();
    e1 = c.prof->get();
    cudaEventRecord(e0, c.s);
    Prof::Rec& r = c.prof->recs[name];
    r.a.push_back(e0);
    r.bytes += bytes;
    r.bytes_stored += stored < 0.0 ? bytes : stored;
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(e1, c.s);
    c.prof->recs[name].b.push_back(e1);
  }
};

// Adds algorithmic bytes to the record of `name` when the name is being profiled (for work whose
// size is known only after its launches were issued).
inline void prof_add_bytes(Ctx& c, const char* name, double bytes) {
  if (c.prof && c.prof->wants(name)) {
    c.prof->recs[name].bytes += bytes;
    c.prof->recs[name].bytes_stored += bytes;
  }
}

void* dev_alloc(Ctx& c, size_t bytes);
void dev_free(Ctx& c, void* p, size_t bytes);

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  Ctx* c = nullptr;
  DBuf() = default;
  DBuf(Ctx& ctx, size_t count) { alloc(ctx, count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), c(o.c) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; c = o.c; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(Ctx& ctx, size_t count) {
    release();
    c = &ctx;
    n = count;
    p = static_cast<T*>(dev_alloc(ctx, (count ? count : 1) * sizeof(T) + 16));  // +16: vector-load slack
  }
  void release() {
    if (p && c) dev_free(*c, p, (n ? n : 1) * sizeof(T) + 16);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
  operator T*() const { return p; }
};

// Device CSR: int64 row pointers, int32 ascending columns.
template <class T>
struct DCSR {
  int64_t nr = 0, nc = 0, nnz = 0;
  DBuf<int64_t> rp;
  DBuf<int32_t> ci;
  DBuf<T> v;
  bool empty() const { return rp.p == nullptr; }
};

// Read back a device scalar (synchronises the stream).
template <class T>
T read_scalar(Ctx& c, const T* dptr) {
  static_assert(sizeof(T) <= 8, "scalar read-backs of at most 8 bytes");
  T h;
  if (c.h_pinned) {  // a copy into pinned memory is a plain DMA: no staging by the driver
    CU(cudaMemcpyAsync(c.h_pinned, dptr, sizeof(T), cudaMemcpyDeviceToHost, c.s));
    CU(cudaStreamSynchronize(c.s));
    memcpy(&h, c.h_pinned, sizeof(T));
  } else {
    CU(cudaMemcpyAsync(&h, dptr, sizeof(T), cudaMemcpyDeviceToHost, c.s));
    CU(cudaStreamSynchronize(c.s));
  }
  ++g_wait_count;
  return h;
}
// Waits for the context's stream (counted in g_wait_count).
inline void host_wait(Ctx& c) {
  CU(cudaStreamSynchronize(c.s));
  ++g_wait_count;
}
// Several device scalars (at most PIN_SLOTS, 8 bytes each at most) read back with one wait.
struct ReadItem {
  const void* src;
  void* dst;
  size_t bytes;
};
inline void read_back(Ctx& c, std::initializer_list<ReadItem> items) {
  if (items.size() > (size_t)PIN_SLOTS) throw Error(MGR_ERR_CUDA, "read_back: too many items");
  char* hp = static_cast<char*>(c.h_pinned);
  size_t k = 0;
  for (const ReadItem& it : items) {
    CU(cudaMemcpyAsync(hp ? hp + 8 * k : it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost, c.s));
    ++k;
  }
  host_wait(c);
  if (hp) {
    k = 0;
    for (const ReadItem& it : items) {
      memcpy(it.dst, hp + 8 * k, it.bytes);
      ++k;
    }
  }
}
void check_errors(Ctx& c, const char* phase);  // reads d_err, throws on set bits, clears it

// Programmatic dependent launch.  A kernel launched by launch_pdl may be scheduled while its
// predecessor in the stream still runs (the launch latency of a chain of short dependent kernels
// overlaps the previous one).  Such a kernel calls pdl_wait() before it touches global memory: it
// returns once the predecessor grid has completed and its writes are visible (at once for a kernel
// launched without the attribute), and then lets the next kernel be scheduled; that kernel can start
// only after every block of this one has passed this point, so all of this grid is resident or done
// by then.
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(Ctx& c, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.pdl ? 1 : 0;
  cuda_check(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...), "kernel launch", __FILE__, __LINE__);
}

inline unsigned grid_for(int64_t n, int block, int64_t cap = (1ll << 30)) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------------------------
// Device helpers.
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  // first position in [lo, hi) with a[pos] >= key
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if (a[m] < key) lo = m + 1; else hi = m;
  }
  return lo;
}
__device__ __forceinline__ int64_t find_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  int64_t p = lower_bound_i32(a, lo, hi, key);
  return (p < hi && a[p] == key) ? p : -1;
}

// 16-byte asynchronous global->shared copy (cp.async, L2 only) and its completion wait.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Row copies by groups of RG lanes (a warp takes 32 / RG rows): lane g of a group takes entries g,
// g + RG, ... of its row, and the output position of an entry is its row's running offset plus the
// number of lower lanes of its group that write in the same round (a ballot masked to the group), so
// a round writes RG consecutive entries of a row instead of one entry of each of 32 rows.
constexpr int RG = 8;
struct RowGroup {
  int g;           // lane within the group
  unsigned gmask;  // the group's lanes
  unsigned below;  // the group's lanes below this one
};
__device__ __forceinline__ RowGroup row_group() {
  const int lane = threadIdx.x & 31;
  RowGroup r;
  r.g = lane & (RG - 1);
  r.gmask = ((1u << RG) - 1u) << (lane & ~(RG - 1));
  r.below = r.gmask & ((1u << lane) - 1u);
  return r;
}
__device__ __forceinline__ int warp_max_int(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------------
// Scans (scan.cu).  out has n+1 entries: out[0] = 0, out[i+1] = sum_{j<=i} in[j].
void scan_excl_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n);
void scan_excl_i32(Ctx& c, const int32_t* in, int32_t* out, int64_t n);
// Build rowptr from per-row counts (int64) and return the total (synchronises).
int64_t counts_to_rowptr(Ctx& c, const int64_t* counts, int64_t* rowptr, int64_t n);
void fill_i64(Ctx& c, int64_t* p, int64_t v, int64_t n);
void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n);
void fill_f64(Ctx& c, double* p, double v, int64_t n);

// ---------------------------------------------------------------------------------------------
// Sparse setup primitives (sparse.cu).  All FP64, deterministic, no fused multiply-add.
void bsr3_validate(Ctx& c, const mgr_bsr3_t& A, const int8_t* marker);  // throws INVALID_ARG
// the host checks and the device check, whose error bits the caller reads (check_errors) before any
// kernel indexes with the pattern
void bsr3_validate_launch(Ctx& c, const mgr_bsr3_t& A, const int8_t* marker);
void bsr3_to_csr(Ctx& c, const mgr_bsr3_t& A, DCSR<double>& out);        // exact zeros dropped
void bsr3_block_inverse(Ctx& c, const mgr_bsr3_t& A, double* binv);      // sets EBIT_SINGULAR
// C = A * B: structural pattern, each entry summed in ascending intermediate index.
// C = A B (Gustavson order); `name` labels the call in the per-kernel timing
// C = A B in Gustavson's order (every entry summed from 0.0 in ascending intermediate index).
// sort_rows: rows of 33..256 products are formed by a warp sort of their products rather than a
// hash table (measured faster for the injective-R coarse operators A_C P of the second and third
// reductions, slower for the first reduction's and the AMG products).
void spgemm(Ctx& c, const DCSR<double>& A, const DCSR<double>& B, DCSR<double>& C, const char* name = "spgemm",
            bool sort_rows = false);
// Pattern of C = A * B only (values left unallocated), same pattern rules.
void transpose(Ctx& c, const DCSR<double>& A, DCSR<double>& T);          // rows sorted by column
// Sort each row segment [rp[i], rp[i+1]) of (ci, v) by ci (keys unique within a row).
void sort_rows(Ctx& c, int64_t nr, const int64_t* rp, int32_t* ci, double* v);

// CSR float copy
void csr_to_f32(Ctx& c, const DCSR<double>& A, DCSR<float>& B);
void copy_csr(Ctx& c, const DCSR<double>& A, DCSR<double>& B);
// B = the rows `rows` of A; nnz >= 0: B's entry count, known to the caller (no read-back)
void csr_gather_rows(Ctx& c, const DCSR<double>& A, const int32_t* rows, int64_t nr, DCSR<double>& B,
                     int64_t nnz = -1);

}  // namespace mgr
