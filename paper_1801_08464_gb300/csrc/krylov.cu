// krylov.cu -- FP64 kernels of the flexible GMRES outer iteration (section 6: GMRES around the
// MGR preconditioner) and of the adjoint helpers: BSR SpMV, deterministic multi-dot products with
// warp-shuffle reductions, Gram-Schmidt updates, solution update, block transpose, outer-product
// gradient.  Reductions are two-stage with a fixed grid, so results do not depend on timing.
#include <array>
#include <map>
#include <mutex>

#include "apply.cuh"

namespace mgr {

// y = A x or y = sub - A x, one thread per block row
__global__ void __launch_bounds__(256) k_bsr3_spmv_f64(int64_t nb, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ x, const double* __restrict__ sub,
                                                       double* __restrict__ y) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int64_t k1 = rp[I + 1];
  for (int64_t k = rp[I]; k < k1; ++k) {
    int64_t J = ci[k];
    const double* b = v + 9 * k;
    double x0 = __ldg(x + 3 * J), x1 = __ldg(x + 3 * J + 1), x2 = __ldg(x + 3 * J + 2);
    s0 = fma(b[0], x0, s0); s0 = fma(b[1], x1, s0); s0 = fma(b[2], x2, s0);
    s1 = fma(b[3], x0, s1); s1 = fma(b[4], x1, s1); s1 = fma(b[5], x2, s1);
    s2 = fma(b[6], x0, s2); s2 = fma(b[7], x1, s2); s2 = fma(b[8], x2, s2);
  }
  if (sub) { s0 = sub[3 * I] - s0; s1 = sub[3 * I + 1] - s1; s2 = sub[3 * I + 2] - s2; }
  y[3 * I] = s0;
  y[3 * I + 1] = s1;
  y[3 * I + 2] = s2;
}

struct EpiSpmvF64 {  // y = A x, or y = sub - A x
  const double* sub;
  double* y;
  __device__ void operator()(int64_t I, double s0, double s1, double s2) const {
    if (sub) { s0 = sub[3 * I] - s0; s1 = sub[3 * I + 1] - s1; s2 = sub[3 * I + 2] - s2; }
    y[3 * I] = s0;
    y[3 * I + 1] = s1;
    y[3 * I + 2] = s2;
  }
};

void launch_bsr3_spmv_f64(Ctx& c, const mgr_bsr3_t& A, const double* x, const double* sub, double* y) {
  launch_pdl(c, k_bsr3_spmv_f64, grid_for(A.nb, 256), 256, 0, A.nb, A.rowptr, A.colind, A.values, x, sub, y);
  CU_LAUNCH();
}

void launch_sell_spmv_f64(Ctx& c, const SellPattern& S, const double* vals, const double* x, const double* sub,
                          double* y) {
  // values, block columns, row pointers, x, y (and the subtrahend)
  ProfScope ps(c, "bsr3_spmv_f64", 76.0 * S.nnzb_real + 8.0 * (S.nb + 1) + 48.0 * S.nb + (sub ? 24.0 * S.nb : 0.0));
  launch_bsr_sell<double, double>(c, S, vals, x, EpiSpmvF64{sub, y});
}

// ---- multi-dot ---------------------------------------------------------------------------------
constexpr int KT = 256;
constexpr int MD_BLOCKS = 1216;  // upper bound of the one-wave grids below (8 blocks per SM on 152 SMs)

template <int NA>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NA], int na, double* part) {
  __shared__ double sh[KT / 32][NA];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    if (k < na) {
      double v = warp_sum(acc[k]);
      if (lane == 0) sh[wid][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < na) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += sh[w][threadIdx.x];
    part[(int64_t)blockIdx.x * na + threadIdx.x] = s;
  }
}

// Sums of NA per-thread values over the block (KT threads), thread t < NA ending with sum t.  Within a
// warp a reduce-scatter: each step keeps half of the values and adds the partner lane's copy of that
// half (P = 32 values cost 31 FP64 additions per lane, a shuffle tree per value 160); a shuffle tree
// per value when NA is small.
template <int NA>
__device__ __forceinline__ double block_reduce_many(const double (&acc)[NA]) {
  __shared__ double red[KT / 32][NA];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (NA * 5 <= 31) {
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const double v = warp_sum(acc[k]);
      if (lane == 0) red[wid][k] = v;
    }
  } else {
    constexpr int P = NA <= 32 ? 32 : 64;
    double v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = k < NA ? acc[k] : 0.0;
#pragma unroll
    for (int o = 16, c = P; o >= 1; o >>= 1, c >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < c / 2; ++j) {
        const double lo = v[j], hi = v[j + c / 2];
        const double send = up ? lo : hi;
        const double keep = up ? hi : lo;
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    // lane L now holds the warp sums of values (P/32) L + j, j < P/32
#pragma unroll
    for (int j = 0; j < P / 32; ++j) {
      const int k = (P / 32) * lane + j;
      if (k < NA) red[wid][k] = v[j];
    }
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < NA) {
#pragma unroll
    for (int q = 0; q < KT / 32; ++q) s += red[q][threadIdx.x];
  }
  return s;
}

// Multi-dot in one pass over the rows: every thread takes pairs of rows and all NV vectors at once
// (w read once, one FMA per product, one instantiation per vector count so the k loop is unrolled
// whole), grid-stride over one resident wave.  Staging the tiles through shared memory with bulk
// copies, or prefetching the next pair into registers, measured slower: the FP64 pipe, not the
// loads, sets the pace.  With ww, acc[NV] takes w . w.  Partials: part[k * gridDim.x + x] (a second
// launch adds them up; the last block doing it in place measured slower, since its serial sum over
// the blocks' partials is on the critical path).
template <int NV>
__global__ void __launch_bounds__(KT) k_mdot(int64_t n, const double* __restrict__ V, int64_t ldv,
                                             const double* __restrict__ w, int ww, double* __restrict__ part) {
  pdl_wait();
  double acc[NV + 1];
#pragma unroll
  for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
  const int64_t n2 = n >> 1;
  // pairs of doubles: V, w 16-byte aligned and ldv even, so every pair is aligned
  for (int64_t q = blockIdx.x * (int64_t)KT + threadIdx.x; q < n2; q += (int64_t)gridDim.x * KT) {
    const int64_t i = 2 * q;
    const double2 wi = *reinterpret_cast<const double2*>(w + i);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(V + k * ldv + i));
      acc[k] = fma(v.x, wi.x, acc[k]);
      acc[k] = fma(v.y, wi.y, acc[k]);
    }
    if (ww) {
      acc[NV] = fma(wi.x, wi.x, acc[NV]);
      acc[NV] = fma(wi.y, wi.y, acc[NV]);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(V[k * ldv + i], wi, acc[k]);
    if (ww) acc[NV] = fma(wi, wi, acc[NV]);
  }
  const double s = block_reduce_many<NV + 1>(acc);
  const int t = threadIdx.x;
  if (t < NV || (t == NV && ww)) part[(int64_t)t * gridDim.x + blockIdx.x] = s;
}

using MdotFn = void (*)(int64_t, const double*, int64_t, const double*, int, double*);
template <int... I>
constexpr std::array<MdotFn, sizeof...(I)> mdot_table(std::integer_sequence<int, I...>) {
  return {k_mdot<I + 1>...};
}
static const std::array<MdotFn, KRY_MAXV> kMdot = mdot_table(std::make_integer_sequence<int, KRY_MAXV>{});

// out[k] = sum over the nx partials of k, in a fixed order (a warp per k, strided lanes, then a
// fixed shuffle tree)
__global__ void k_reduce_parts(int nx, int na, const double* __restrict__ part, double* __restrict__ out) {
  pdl_wait();
  int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (k >= na) return;
  double s = 0.0;
  for (int x = lane; x < nx; x += 32) s += part[(int64_t)k * nx + x];
  s = warp_sum(s);
  if (lane == 0) out[k] = s;
}

// Blocks of `fn` (KT threads, static shared memory only) resident on the whole device at once, at
// most MD_BLOCKS: streaming kernels launch exactly one full wave, with no partial second wave.
static int one_wave(const void* fn) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, fn);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, sms = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, KT, 0));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int nb = per_sm * sms;
  if (nb < 1) nb = 1;
  if (nb > MD_BLOCKS) nb = MD_BLOCKS;
  cache[key] = nb;
  return nb;
}

void launch_mdot(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* w, bool want_ww, double* part,
                 double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "multi-dot with more than 32 vectors");
  const int ww = want_ww ? 1 : 0;
  ProfScope ps(c, "mdot", 8.0 * (nv + 1) * n);
  if (nv < 1) {  // w . w alone
    launch_nrm2sq(c, n, w, part, out);
    return;
  }
  const MdotFn fn = kMdot[nv - 1];
  const int nx = one_wave((const void*)fn);
  launch_pdl(c, fn, nx, KT, 0, n, V, ldv, w, ww, part);
  CU_LAUNCH();
  const int na = nv + ww;
  launch_pdl(c, k_reduce_parts, (na + 7) / 8, 256, 0, nx, na, part, out);
  CU_LAUNCH();
}

// v_out = s (w - sum_k h[k] V_k) (h and s read from device memory; s == nullptr means 1), and
// ||v_out||^2 partials when part != nullptr.  v_out may alias w.  NV > 0: the vector count nv is the
// compile-time NV and the k loop is unrolled whole (no remainder loop that waits for one load at a
// time); NV = 0 takes nv at run time.  Each entry subtracts its products in ascending k either way.
// NORM: the squared norm is accumulated (an FMA per entry, which the FP64 pipe pays for) only when
// it is wanted.
template <int NV, bool NORM>
__global__ void __launch_bounds__(KT) k_mupdate(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                                                const double* __restrict__ h, const double* __restrict__ sp,
                                                const double* w, double* vout, double* __restrict__ part) {
  pdl_wait();
  const int cnt = NV > 0 ? NV : nv;
  __shared__ double sh_h[KRY_MAXV];
  if (threadIdx.x < cnt) sh_h[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double sc = sp ? *sp : 1.0;
  double acc[1] = {0.0};
  int64_t n2 = n >> 1;
  for (int64_t q = blockIdx.x * (int64_t)KT + threadIdx.x; q < n2; q += (int64_t)gridDim.x * KT) {
    int64_t i = 2 * q;
    double2 s = *reinterpret_cast<const double2*>(w + i);
    if constexpr (NV > 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double2 v = __ldg(reinterpret_cast<const double2*>(V + k * ldv + i));
        s.x -= sh_h[k] * v.x;
        s.y -= sh_h[k] * v.y;
      }
    } else {
#pragma unroll 8
      for (int k = 0; k < nv; ++k) {
        double2 v = __ldg(reinterpret_cast<const double2*>(V + k * ldv + i));
        s.x -= sh_h[k] * v.x;
        s.y -= sh_h[k] * v.y;
      }
    }
    s.x *= sc;
    s.y *= sc;
    *reinterpret_cast<double2*>(vout + i) = s;
    if (NORM) {
      acc[0] = fma(s.x, s.x, acc[0]);
      acc[0] = fma(s.y, s.y, acc[0]);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t i = n - 1;
    double s = w[i];
    for (int k = 0; k < cnt; ++k) s -= sh_h[k] * V[k * ldv + i];
    s *= sc;
    vout[i] = s;
    acc[0] += s * s;
  }
  if (NORM) block_reduce_store<1>(acc, 1, part);
}

using MupdateFn = void (*)(int64_t, const double*, int64_t, int, const double*, const double*, const double*, double*,
                           double*);
template <bool NORM, int... I>
constexpr std::array<MupdateFn, sizeof...(I)> mupdate_table(std::integer_sequence<int, I...>) {
  return {k_mupdate<I, NORM>...};
}
static const std::array<MupdateFn, KRY_MAXV + 1> kMupdate[2] = {
    mupdate_table<false>(std::make_integer_sequence<int, KRY_MAXV + 1>{}),
    mupdate_table<true>(std::make_integer_sequence<int, KRY_MAXV + 1>{})};

void launch_mupdate(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* h, const double* scale,
                    const double* w, double* vout, double* part, double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "update with more than 32 vectors");
  ProfScope ps(c, "mupdate", 8.0 * (nv + 2) * n);
  const MupdateFn fn = kMupdate[out ? 1 : 0][nv > 0 ? nv : 0];
  const int grid = one_wave((const void*)fn);
  launch_pdl(c, fn, grid, KT, 0, n, V, ldv, nv, h, scale, w, vout, out ? part : nullptr);
  CU_LAUNCH();
  if (out) {
    launch_pdl(c, k_reduce_parts, 1, 32, 0, grid, 1, part, out);
    CU_LAUNCH();
  }
}

// s_out = 1 / sqrt(ww - sum_k h_k^2): the Pythagorean norm of w - V h for orthonormal V
__global__ void k_pyth_scale(int nv, const double* __restrict__ h, const double* __restrict__ ww, double* out) {
  pdl_wait();
  if (threadIdx.x != 0) return;
  double s = *ww;
  for (int k = 0; k < nv; ++k) s -= h[k] * h[k];
  out[0] = s;                          // squared norm (for the host)
  out[1] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
}
void launch_pyth_scale(Ctx& c, int nv, const double* h, const double* ww, double* out) {
  launch_pdl(c, k_pyth_scale, 1, 32, 0, nv, h, ww, out);
  CU_LAUNCH();
}

__global__ void __launch_bounds__(KT) k_nrm2sq(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  pdl_wait();
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) acc[0] += x[i] * x[i];
  block_reduce_store<1>(acc, 1, part);
}
void launch_nrm2sq(Ctx& c, int64_t n, const double* x, double* part, double* out) {
  launch_pdl(c, k_nrm2sq, KRY_GRID, KT, 0, n, x, part);
  CU_LAUNCH();
  launch_pdl(c, k_reduce_parts, 1, 32, 0, KRY_GRID, 1, part, out);
  CU_LAUNCH();
}

__global__ void k_scal(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
void launch_scal(Ctx& c, int64_t n, double alpha, const double* x, double* y) {
  launch_pdl(c, k_scal, grid_for(n, 256, 4 * 1024), 256, 0, n, alpha, x, y);
  CU_LAUNCH();
}

// x += Z y (one solution update per restart cycle): pairs of doubles per thread, one resident wave,
// each entry's FMAs in ascending k as before; a misaligned x takes the scalar form
__global__ void __launch_bounds__(KT) k_xupdate(int64_t n, const double* __restrict__ Z, int64_t ldz, int nz,
                                                const double* __restrict__ y, double* __restrict__ x, int vec) {
  pdl_wait();
  __shared__ double sy[KRY_MAXV];
  if (threadIdx.x < nz) sy[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  if (vec) {
    const int64_t n2 = n >> 1;
    for (int64_t q = blockIdx.x * (int64_t)KT + threadIdx.x; q < n2; q += (int64_t)gridDim.x * KT) {
      const int64_t i = 2 * q;
      double2 s = *reinterpret_cast<const double2*>(x + i);
#pragma unroll 8
      for (int k = 0; k < nz; ++k) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(Z + k * ldz + i));
        s.x = fma(sy[k], v.x, s.x);
        s.y = fma(sy[k], v.y, s.y);
      }
      *reinterpret_cast<double2*>(x + i) = s;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
      const int64_t i = n - 1;
      double s = x[i];
      for (int k = 0; k < nz; ++k) s = fma(sy[k], Z[k * ldz + i], s);
      x[i] = s;
    }
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int k = 0; k < nz; ++k) s = fma(sy[k], Z[k * ldz + i], s);
    x[i] = s;
  }
}
void launch_xupdate(Ctx& c, int64_t n, const double* Z, int64_t ldz, int nz, const double* y, double* x) {
  const int vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(Z)) & 15) == 0 && (ldz & 1) == 0;
  const int grid = one_wave((const void*)k_xupdate);
  for (int k0 = 0; k0 < nz; k0 += KRY_MAXV) {
    int m = nz - k0 < KRY_MAXV ? nz - k0 : KRY_MAXV;
    launch_pdl(c, k_xupdate, grid, KT, 0, n, Z + k0 * ldz, ldz, m, y + k0, x, vec);
    CU_LAUNCH();
  }
}

// ---- adjoint helpers ---------------------------------------------------------------------------
// g[9k + 3p + q] = -lam[3I+p] x[3J+q]
__global__ void k_outer_grad(int64_t nb, const int64_t* rp, const int32_t* ci, const double* lam, const double* x,
                             double* g) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  double l0 = lam[3 * I], l1 = lam[3 * I + 1], l2 = lam[3 * I + 2];
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
    int64_t J = ci[k];
    double x0 = x[3 * J], x1 = x[3 * J + 1], x2 = x[3 * J + 2];
    double* o = g + 9 * k;
    o[0] = -l0 * x0; o[1] = -l0 * x1; o[2] = -l0 * x2;
    o[3] = -l1 * x0; o[4] = -l1 * x1; o[5] = -l1 * x2;
    o[6] = -l2 * x0; o[7] = -l2 * x1; o[8] = -l2 * x2;
  }
}
void launch_bsr3_outer_grad(Ctx& c, const mgr_bsr3_t& A, const double* lam, const double* x, double* g) {
  launch_pdl(c, k_outer_grad, grid_for(A.nb, 256), 256, 0, A.nb, A.rowptr, A.colind, lam, x, g);
  CU_LAUNCH();
}

__global__ void k_bcol_count(int64_t nnzb, const int32_t* ci, unsigned long long* cnt) {
  pdl_wait();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[k]], 1ull);
}
__global__ void k_bscatter(int64_t nb, const int64_t* rp, const int32_t* ci, const int64_t* trp, unsigned long long* slot,
                           int32_t* tci, int64_t* src) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
    int32_t J = ci[k];
    int64_t d = trp[J] + (int64_t)atomicAdd(&slot[J], 1ull);
    tci[d] = (int32_t)I;
    src[d] = k;
  }
}
// sort each transposed block row by column (insertion sort: block rows are short), then copy the
// transposed 3x3 blocks
__global__ void k_bsort_fill(int64_t nb, const int64_t* trp, int32_t* tci, int64_t* src, const double* v, double* vt) {
  pdl_wait();
  int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (J >= nb) return;
  int64_t b = trp[J], e = trp[J + 1];
  for (int64_t a = b + 1; a < e; ++a) {
    int32_t key = tci[a];
    int64_t s = src[a];
    int64_t t = a - 1;
    while (t >= b && tci[t] > key) { tci[t + 1] = tci[t]; src[t + 1] = src[t]; --t; }
    tci[t + 1] = key;
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
void launch_bsr3_transpose(Ctx& c, const mgr_bsr3_t& A, int64_t* rpt, int32_t* cit, double* vt) {
  DBuf<unsigned long long> cnt(c, A.nb + 1);
  DBuf<int64_t> src(c, A.nnzb);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  launch_pdl(c, k_bcol_count, grid_for(A.nnzb, 256, 8192), 256, 0, A.nnzb, A.colind, cnt.p);
  CU_LAUNCH();
  scan_excl_i64(c, reinterpret_cast<const int64_t*>(cnt.p), rpt, A.nb);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  launch_pdl(c, k_bscatter, grid_for(A.nb, 256), 256, 0, A.nb, A.rowptr, A.colind, rpt, cnt.p, cit, src.p);
  CU_LAUNCH();
  launch_pdl(c, k_bsort_fill, grid_for(A.nb, 256), 256, 0, A.nb, rpt, cit, src.p, A.values, vt);
  CU_LAUNCH();
  CU(cudaStreamSynchronize(c.s));
}

// Pattern of A^T (row pointers, block columns ascending) and, per transposed block, the index of its
// source block in A.
__global__ void k_bsort_src(int64_t nb, const int64_t* trp, int32_t* tci, int64_t* src) {
  pdl_wait();
  int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (J >= nb) return;
  int64_t b = trp[J], e = trp[J + 1];
  for (int64_t a = b + 1; a < e; ++a) {
    int32_t key = tci[a];
    int64_t s = src[a];
    int64_t t = a - 1;
    while (t >= b && tci[t] > key) { tci[t + 1] = tci[t]; src[t + 1] = src[t]; --t; }
    tci[t + 1] = key;
    src[t + 1] = s;
  }
}
void launch_bsr3_transpose_pattern(Ctx& c, const mgr_bsr3_t& A, int64_t* rpt, int32_t* cit, int64_t* src) {
  DBuf<unsigned long long> cnt(c, A.nb + 1);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  launch_pdl(c, k_bcol_count, grid_for(A.nnzb, 256, 8192), 256, 0, A.nnzb, A.colind, cnt.p);
  CU_LAUNCH();
  scan_excl_i64(c, reinterpret_cast<const int64_t*>(cnt.p), rpt, A.nb);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  launch_pdl(c, k_bscatter, grid_for(A.nb, 256), 256, 0, A.nb, A.rowptr, A.colind, rpt, cnt.p, cit, src);
  CU_LAUNCH();
  launch_pdl(c, k_bsort_src, grid_for(A.nb, 256), 256, 0, A.nb, rpt, cit, src);
  CU_LAUNCH();
}

}  // namespace mgr
