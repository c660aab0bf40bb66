// krylov.cu -- FP64 kernels of the flexible GMRES outer iteration (section 6: GMRES around the
// MGR preconditioner) and of the adjoint helpers: BSR SpMV, deterministic multi-dot products with
// warp-shuffle reductions, Gram-Schmidt updates, solution update, block transpose, outer-product
// gradient.  Reductions are two-stage with a fixed grid, so results do not depend on timing.
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
constexpr int MD_VEC = 8;        // vectors per block column of the 2-D multi-dot grid
constexpr int MD_BLOCKS = 1216;  // upper bound of the grids below (8 blocks per SM on 152 SMs)

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

// The products of one block: KN vectors (KN <= MD_VEC, a compile-time count, so no FMA of a vector the
// block does not hold is issued, not even predicated off) and, with DOW, w . w as well.
template <int KN, bool DOW>
__device__ __forceinline__ void mdot_rows(int64_t i0, int64_t i1, const double* __restrict__ V, int64_t ldv,
                                          const double* __restrict__ w, double (&acc)[MD_VEC + 1]) {
  // pairs of doubles: chunk is even and ldv is even, so every pair is 16-byte aligned
  for (int64_t i = i0 + 2 * threadIdx.x; i < i1; i += 2 * KT) {
    if (i + 1 < i1) {
      double2 wi = *reinterpret_cast<const double2*>(w + i);
      // one FMA per product: FP64 instructions, not bytes, bound this kernel on this GPU
#pragma unroll
      for (int k = 0; k < KN; ++k) {
        double2 v = __ldg(reinterpret_cast<const double2*>(V + k * ldv + i));
        acc[k] = fma(v.x, wi.x, acc[k]);
        acc[k] = fma(v.y, wi.y, acc[k]);
      }
      if (DOW) {
        acc[MD_VEC] = fma(wi.x, wi.x, acc[MD_VEC]);
        acc[MD_VEC] = fma(wi.y, wi.y, acc[MD_VEC]);
      }
    } else {
      double wi = w[i];
#pragma unroll
      for (int k = 0; k < KN; ++k) acc[k] = fma(V[k * ldv + i], wi, acc[k]);
      if (DOW) acc[MD_VEC] = fma(wi, wi, acc[MD_VEC]);
    }
  }
}

template <bool DOW>
__device__ __forceinline__ void mdot_rows_kn(int kn, int64_t i0, int64_t i1, const double* __restrict__ V,
                                             int64_t ldv, const double* __restrict__ w, double (&acc)[MD_VEC + 1]) {
  static_assert(MD_VEC == 8, "one case per vector count of a block");
  switch (kn) {
    case 0: mdot_rows<0, DOW>(i0, i1, V, ldv, w, acc); break;  // w . w alone
    case 1: mdot_rows<1, DOW>(i0, i1, V, ldv, w, acc); break;
    case 2: mdot_rows<2, DOW>(i0, i1, V, ldv, w, acc); break;
    case 3: mdot_rows<3, DOW>(i0, i1, V, ldv, w, acc); break;
    case 4: mdot_rows<4, DOW>(i0, i1, V, ldv, w, acc); break;
    case 5: mdot_rows<5, DOW>(i0, i1, V, ldv, w, acc); break;
    case 6: mdot_rows<6, DOW>(i0, i1, V, ldv, w, acc); break;
    case 7: mdot_rows<7, DOW>(i0, i1, V, ldv, w, acc); break;
    default: mdot_rows<8, DOW>(i0, i1, V, ldv, w, acc); break;
  }
}

// Multi-dot: block x handles row chunk x for every vector group g (vectors 8g .. 8g+7) in turn, so
// every block streams the same number of vectors (a 2-D grid of group blocks left the blocks of a
// short last group idle for most of the launch).  Group 0 also accumulates w . w.  Partial sums go
// to part[k * nx + x] (k = nv for w . w).
__global__ void __launch_bounds__(KT) k_mdot(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                                             const double* __restrict__ w, int ww, int ng, int nx, int64_t chunk,
                                             double* __restrict__ part) {
  pdl_wait();
  const int x = blockIdx.x;
  const int64_t i0 = (int64_t)x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
  __shared__ double sh[KT / 32][MD_VEC + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = 0; g < ng; ++g) {
    const int k0 = g * MD_VEC;
    const int kn = nv - k0 < MD_VEC ? nv - k0 : MD_VEC;
    const bool dow = ww && g == 0;
    double acc[MD_VEC + 1];
#pragma unroll
    for (int k = 0; k <= MD_VEC; ++k) acc[k] = 0.0;
    // kn and dow are uniform over the block
    if (dow) mdot_rows_kn<true>(kn, i0, i1, V + k0 * ldv, ldv, w, acc);
    else mdot_rows_kn<false>(kn, i0, i1, V + k0 * ldv, ldv, w, acc);
    // reduce-scatter of the 8 vector sums across the warp (FP64 adds are the scarce instructions): at
    // offsets 16, 8, 4 each lane keeps half of its values and adds its partner's copy of that half
    // (4 + 2 + 1 adds), then a butterfly over offsets 2 and 1; lane L ends with the warp's sum of
    // vector ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1).  9 adds instead of 40.
    {
      static_assert(MD_VEC == 8, "the reduce-scatter is written for 8 vectors per block");
      double h4[4], h2[2], h1;
      const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double send = b16 ? acc[j] : acc[j + 4];
        double keep = b16 ? acc[j + 4] : acc[j];
        h4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        double send = b8 ? h4[j] : h4[j + 2];
        double keep = b8 ? h4[j + 2] : h4[j];
        h2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
      {
        double send = b4 ? h2[0] : h2[1];
        double keep = b4 ? h2[1] : h2[0];
        h1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
      h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
      if ((lane & 3) == 0) sh[wid][(b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0)] = h1;
      if (dow) {  // uniform over the block
        double v = warp_sum(acc[MD_VEC]);
        if (lane == 0) sh[wid][MD_VEC] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x <= MD_VEC) {
      int k = threadIdx.x;
      if (k < kn || (k == MD_VEC && dow)) {
        double s = 0.0;
        for (int w2 = 0; w2 < KT / 32; ++w2) s += sh[w2][k];
        int out = (k == MD_VEC) ? nv : k0 + k;
        part[(int64_t)out * nx + x] = s;
      }
    }
    __syncthreads();  // sh is reused by the next group
  }
}

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

static int md_nx(int64_t n, int64_t* chunk) {
  int nx = one_wave((const void*)k_mdot);
  if (nx < 1) nx = 1;
  int64_t c = (n + nx - 1) / nx;
  c = (c + 1) & ~int64_t(1);
  if (c < 2 * KT) c = 2 * KT;
  *chunk = c;
  return (int)((n + c - 1) / c);
}

void launch_mdot(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* w, bool want_ww, double* part,
                 double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "multi-dot with more than 32 vectors");
  int ww = want_ww ? 1 : 0;
  int ng = (nv + MD_VEC - 1) / MD_VEC;
  if (ng < 1) ng = 1;
  int64_t chunk;
  int nx = md_nx(n, &chunk);
  ProfScope ps(c, "mdot", 8.0 * (nv + 1) * n);
  launch_pdl(c, k_mdot, nx, KT, 0, n, V, ldv, nv, w, ww, ng, nx, chunk, part);
  CU_LAUNCH();
  int na = nv + ww;
  launch_pdl(c, k_reduce_parts, (na + 7) / 8, 256, 0, nx, na, part, out);
  CU_LAUNCH();
}

// v_out = s (w - sum_k h[k] V_k) (h and s read from device memory; s == nullptr means 1), and
// ||v_out||^2 partials when part != nullptr.  v_out may alias w.  NV > 0: the vector count nv is the
// compile-time NV and the k loop is unrolled whole (no remainder loop that waits for one load at a
// time); NV = 0 takes nv at run time.  Each entry subtracts its products in ascending k either way.
template <int NV>
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
    acc[0] = fma(s.x, s.x, acc[0]);
    acc[0] = fma(s.y, s.y, acc[0]);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t i = n - 1;
    double s = w[i];
    for (int k = 0; k < cnt; ++k) s -= sh_h[k] * V[k * ldv + i];
    s *= sc;
    vout[i] = s;
    acc[0] += s * s;
  }
  if (part) block_reduce_store<1>(acc, 1, part);
}

using MupdateFn = void (*)(int64_t, const double*, int64_t, int, const double*, const double*, const double*, double*,
                           double*);
static const MupdateFn kMupdate[KRY_MAXV + 1] = {k_mupdate<0>, k_mupdate<1>, k_mupdate<2>, k_mupdate<3>, k_mupdate<4>, k_mupdate<5>, k_mupdate<6>, k_mupdate<7>, k_mupdate<8>, k_mupdate<9>, k_mupdate<10>, k_mupdate<11>, k_mupdate<12>, k_mupdate<13>, k_mupdate<14>, k_mupdate<15>, k_mupdate<16>, k_mupdate<17>, k_mupdate<18>, k_mupdate<19>, k_mupdate<20>, k_mupdate<21>, k_mupdate<22>, k_mupdate<23>, k_mupdate<24>, k_mupdate<25>, k_mupdate<26>, k_mupdate<27>, k_mupdate<28>, k_mupdate<29>, k_mupdate<30>, k_mupdate<31>, k_mupdate<32>};

void launch_mupdate(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* h, const double* scale,
                    const double* w, double* vout, double* part, double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "update with more than 32 vectors");
  ProfScope ps(c, "mupdate", 8.0 * (nv + 2) * n);
  const MupdateFn fn = kMupdate[nv > 0 ? nv : 0];
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
