// apply.cu -- kernels of one MGR preconditioner application (section 4 Algorithm, section 5
// reduction order) and of the AMG V-cycle used as the coarse solve.  Templated on the working
// precision T (double, or float for the FP32 hierarchy); inputs and outputs at the finest level are
// FP64.  All are memory-bound sparse / vector kernels (no tensor cores).
#include "apply.cuh"
#include "bsr_sell.cuh"

namespace mgr {

template <class T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// ============================== level 0: 3x3 blocks =============================================
template <class T>
__global__ void k_global_relax(int64_t nb, const T* __restrict__ binv, const double* __restrict__ r, T* __restrict__ e0) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  T r0 = (T)r[3 * I], r1 = (T)r[3 * I + 1], r2 = (T)r[3 * I + 2];
  const T* b = binv + 9 * I;
  e0[3 * I + 0] = b[0] * r0 + b[1] * r1 + b[2] * r2;
  e0[3 * I + 1] = b[3] * r0 + b[4] * r1 + b[5] * r2;
  e0[3 * I + 2] = b[6] * r0 + b[7] * r1 + b[8] * r2;
}

template <class T>
void launch_global_relax(Ctx& c, int64_t nb, const T* binv, const double* r, T* e0) {
  ProfScope ps(c, "global_relax", (double)nb * (9 * sizeof(T) + 24 + 3 * sizeof(T)));
  launch_pdl(c, k_global_relax<T>, grid_for(nb, 256), 256, 0, nb, binv, r, e0);
  CU_LAUNCH();
}

// One thread per block row: res_p = r_p - sum_k B_k[p][:] e0[3 J_k + :], routed by map.
template <class T>
__global__ void __launch_bounds__(256) k_bsr_resid_split(int64_t nb, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci, const T* __restrict__ v,
                                                         const double* __restrict__ r, const T* __restrict__ e0,
                                                         const int32_t* __restrict__ map, T* __restrict__ rnext,
                                                         T* __restrict__ resF) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  T s0 = 0, s1 = 0, s2 = 0;
  if (e0) {
    int64_t k0 = rp[I], k1 = rp[I + 1];
    for (int64_t k = k0; k < k1; ++k) {
      int64_t J = ci[k];
      const T* b = v + 9 * k;
      T x0 = ldg(e0 + 3 * J), x1 = ldg(e0 + 3 * J + 1), x2 = ldg(e0 + 3 * J + 2);
      s0 += b[0] * x0 + b[1] * x1 + b[2] * x2;
      s1 += b[3] * x0 + b[4] * x1 + b[5] * x2;
      s2 += b[6] * x0 + b[7] * x1 + b[8] * x2;
    }
  }
  T res[3] = {(T)r[3 * I] - s0, (T)r[3 * I + 1] - s1, (T)r[3 * I + 2] - s2};
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    int32_t m = map[3 * I + p];
    if (m >= 0) rnext[m] = res[p];
    else resF[-m - 1] = res[p];
  }
}

template <class T>
struct EpiSplit {  // res = r - A e0 routed by map
  const double* r; const int32_t* map; T* rnext; T* resF;
  __device__ void operator()(int64_t I, T s0, T s1, T s2) const {
    T res[3] = {(T)r[3 * I] - s0, (T)r[3 * I + 1] - s1, (T)r[3 * I + 2] - s2};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      int32_t m = map[3 * I + p];
      if (m >= 0) rnext[m] = res[p];
      else resF[-m - 1] = res[p];
    }
  }
};

template <class T>
void launch_bsr_resid_split(Ctx& c, const SellPattern& S, const T* vals, const double* r, const T* e0,
                            const int32_t* map, T* rnext, T* resF) {
  // values, block columns, row pointers, e0, r, map, one output per dof
  ProfScope ps(c, "bsr_resid_split",
               e0 ? (double)S.nnzb_real * (9 * sizeof(T) + 4) + 8.0 * (S.nb + 1) + (double)S.nb * (3 * sizeof(T) + 24 + 12 + 3 * sizeof(T))
                  : (double)S.nb * (24 + 12 + 3 * sizeof(T)));
  if (e0) {
    launch_bsr_sell<T, T>(c, S, vals, e0, EpiSplit<T>{r, map, rnext, resF});
  } else {
    launch_pdl(c, k_bsr_resid_split<T>, grid_for(S.nb, 256), 256, 0, S.nb, nullptr, nullptr, vals, r, e0, map, rnext, resF);
    CU_LAUNCH();
  }
}

// ============================== generic CSR row kernel ==========================================
// TPR lanes per row; partial sums reduced with shuffles inside the lane group; the epilogue gets
// (row, A_row . x).
template <class T, int TPR, class Epi>
__global__ void __launch_bounds__(256) k_rows(int64_t nr, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const T* __restrict__ v, const T* __restrict__ x, Epi epi) {
  pdl_wait();
  int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t r = gt / TPR;
  int sub = (int)(gt % TPR);
  bool ok = r < nr;
  T s = 0;
  typename Epi::Pre pre{};
  if (ok && sub == 0) pre = epi.pre(r);  // the epilogue's loads overlap the row's
  if (ok) {
    int64_t k1 = rp[r + 1];
    for (int64_t k = rp[r] + sub; k < k1; k += TPR) s += v[k] * ldg(x + ci[k]);
  }
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
  if (ok && sub == 0) epi.post(r, s, pre);
}

// Streaming loads of operator values and column codes: read once per pass, so they skip L1 and
// leave it to the x gathers, which the rows of a block share.
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) {
  uint32_t v;
  asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
  uint2 v;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_stream(const int4* p) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

// SELL form: one thread per row, slots walked four at a time (padding slots add 0 * x[0])
template <class T>
struct Quad;
template <>
struct Quad<float> {
  __device__ static __forceinline__ float dot(const float* vp, int4 c, const float* x) {
    float4 v = ld_stream(reinterpret_cast<const float4*>(vp));
    float s = v.x * __ldg(x + c.x);
    s = fmaf(v.y, __ldg(x + c.y), s);
    s = fmaf(v.z, __ldg(x + c.z), s);
    return fmaf(v.w, __ldg(x + c.w), s);
  }
};
template <>
struct Quad<double> {
  __device__ static __forceinline__ double dot(const double* vp, int4 c, const double* x) {
    double2 a = ld_stream(reinterpret_cast<const double2*>(vp));
    double2 b = ld_stream(reinterpret_cast<const double2*>(vp) + 1);
    double s = a.x * __ldg(x + c.x);
    s = fma(a.y, __ldg(x + c.y), s);
    s = fma(b.x, __ldg(x + c.z), s);
    return fma(b.y, __ldg(x + c.w), s);
  }
};

// A 4-slot group of values (streamed) and its product with the four columns given by a word of
// one-byte codes into the table of offsets col - row: the same products in the same order as
// Quad<T>::dot.
template <class T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
  __device__ static __forceinline__ float4 load(const float* p) { return ld_stream(reinterpret_cast<const float4*>(p)); }
  __device__ static __forceinline__ float code_dot(const float4& v, uint32_t raw, int32_t row, const int32_t* tab,
                                                   const float* x) {
    float s = v.x * __ldg(x + row + tab[raw & 0xFFu]);
    s = fmaf(v.y, __ldg(x + row + tab[(raw >> 8) & 0xFFu]), s);
    s = fmaf(v.z, __ldg(x + row + tab[(raw >> 16) & 0xFFu]), s);
    return fmaf(v.w, __ldg(x + row + tab[raw >> 24]), s);
  }
};
template <>
struct Vec4<double> {
  struct type { double2 a, b; };
  __device__ static __forceinline__ type load(const double* p) {
    return {ld_stream(reinterpret_cast<const double2*>(p)), ld_stream(reinterpret_cast<const double2*>(p) + 1)};
  }
  __device__ static __forceinline__ double code_dot(const type& v, uint32_t raw, int32_t row, const int32_t* tab,
                                                    const double* x) {
    double s = v.a.x * __ldg(x + row + tab[raw & 0xFFu]);
    s = fma(v.a.y, __ldg(x + row + tab[(raw >> 8) & 0xFFu]), s);
    s = fma(v.b.x, __ldg(x + row + tab[(raw >> 16) & 0xFFu]), s);
    return fma(v.b.y, __ldg(x + row + tab[raw >> 24]), s);
  }
};

// Column storage of the 4-slot groups: CM 0 = 32-bit indices; 1 = 16-bit offsets from the slice's
// base; 2 = one-byte codes into the operator's table of offsets col - row (held in shared memory),
// laid out in 16-slot groups (rs_code_pos).
struct QuadCols {
  const int32_t* cp;
  const uint16_t* cp16;
  const uint8_t* cp8;
  int32_t base;      // CM 1: the slice's base; CM 2: the row
  const int32_t* tab;  // CM 2: the offsets (shared memory)
  int t;               // CM 2: the row within its slice
};
template <int CM>
__device__ __forceinline__ int4 quad_cols(const QuadCols& qc, int64_t q) {
  if constexpr (CM == 1) {
    const uint2 raw = ld_stream(reinterpret_cast<const uint2*>(qc.cp16 + q * (4 * RS_C)));
    return make_int4(qc.base + (int)(raw.x & 0xFFFFu), qc.base + (int)(raw.x >> 16), qc.base + (int)(raw.y & 0xFFFFu),
                     qc.base + (int)(raw.y >> 16));
  } else if constexpr (CM == 2) {
    const uint32_t raw = ld_stream(reinterpret_cast<const uint32_t*>(qc.cp8 + rs_code_pos(4 * q, qc.t)));
    return make_int4(qc.base + qc.tab[raw & 0xFFu], qc.base + qc.tab[(raw >> 8) & 0xFFu],
                     qc.base + qc.tab[(raw >> 16) & 0xFFu], qc.base + qc.tab[raw >> 24]);
  } else {
    return ld_stream(reinterpret_cast<const int4*>(qc.cp + q * (4 * RS_C)));
  }
}
template <int CM>
__device__ __forceinline__ QuadCols quad_setup(const int32_t* col, const uint16_t* col16, const int32_t* sbase,
                                               const uint8_t* code, const int64_t* coff, const int32_t* tab, int64_t s,
                                               int64_t j0, int t, int64_t row) {
  QuadCols qc{nullptr, nullptr, nullptr, 0, tab, t};
  const int64_t o = j0 * RS_C + t * 4;
  if constexpr (CM == 0) qc.cp = col + o;
  if constexpr (CM == 1) { qc.cp16 = col16 + o; qc.base = sbase[s]; }
  if constexpr (CM == 2) { qc.cp8 = code + coff[s] * RS_C; qc.base = (int32_t)row; }
  return qc;
}

template <class T, class Epi, int Q, int CM>
__global__ void __launch_bounds__(256) k_rows_sell(int64_t nr, const int64_t* __restrict__ soff,
                                                   const int32_t* __restrict__ col, const uint16_t* __restrict__ col16,
                                                   const int32_t* __restrict__ sbase, const uint8_t* __restrict__ code,
                                                   const int64_t* __restrict__ coff,
                                                   const int32_t* __restrict__ otab, const T* __restrict__ val,
                                                   const int32_t* __restrict__ perm, const T* __restrict__ x,
                                                   Epi epi) {
  __shared__ int32_t s_tab[CM == 2 ? 256 : 1];
  pdl_wait();
  if constexpr (CM == 2) {
    if (threadIdx.x < 256) s_tab[threadIdx.x] = otab[threadIdx.x];
    __syncthreads();
  }
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  int64_t s = r / RS_C;
  int t = (int)(r - s * RS_C);
  const int64_t row = perm ? (int64_t)perm[r] : r;
  const typename Epi::Pre pre = epi.pre(row);  // the epilogue's loads overlap the row's
  int64_t j0 = soff[s], nq = (soff[s + 1] - j0) / Q;
  const T* vp = val + j0 * RS_C + t * Q;
  T sum = 0;
  if constexpr (Q == 4 && CM == 2) {
    // one-byte codes: the codes of four groups come in one 16-byte load, then the four groups'
    // values, then their gathers and products (in group order)
    const uint8_t* cb = code + coff[s] * RS_C + t * 16;
    const int32_t r32 = (int32_t)row;
#pragma unroll 1
    for (int64_t q0 = 0; q0 < nq; q0 += 4) {
      const uint4 cw = ld_stream(reinterpret_cast<const uint4*>(cb + q0 * (4 * RS_C)));
      typename Vec4<T>::type vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q0 + u < nq) vv[u] = Vec4<T>::load(vp + (q0 + u) * (4 * RS_C));
      const uint32_t w4[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q0 + u < nq) sum += Vec4<T>::code_dot(vv[u], w4[u], r32, s_tab, x);
    }
  } else if constexpr (Q == 4) {
    const QuadCols qc = quad_setup<CM>(col, col16, sbase, code, coff, s_tab, s, j0, t, row);
#pragma unroll 2
    for (int64_t q = 0; q < nq; ++q) sum += Quad<T>::dot(vp + q * (4 * RS_C), quad_cols<CM>(qc, q), x);
  } else {
    const int32_t* cp = col + j0 * RS_C + t * Q;
#pragma unroll 4
    for (int64_t j = 0; j < nq; ++j) sum += vp[j * RS_C] * ldg(x + cp[j * RS_C]);
  }
  epi.post(row, sum, pre);
}

// SELL form with H threads per row (4-slot groups): thread h of a row takes groups h, h + H, ...;
// the 8 rows of a slice and their H threads are 8H consecutive lanes, so one step of a slice reads
// H consecutive 128-byte lines; partial sums meet by shuffles across lanes 8 and 16 apart.  Used
// when one thread per row would leave the GPU with few waves of long rows (a tail).
template <class T, class Epi, int H, int CM>
__global__ void __launch_bounds__(256) k_rows_sell_split(int64_t nr, const int64_t* __restrict__ soff,
                                                         const int32_t* __restrict__ col,
                                                         const uint16_t* __restrict__ col16,
                                                         const int32_t* __restrict__ sbase,
                                                         const uint8_t* __restrict__ code,
                                                         const int64_t* __restrict__ coff,
                                                         const int32_t* __restrict__ otab, const T* __restrict__ val,
                                                         const int32_t* __restrict__ perm, const T* __restrict__ x,
                                                         Epi epi) {
  __shared__ int32_t s_tab[CM == 2 ? 256 : 1];
  pdl_wait();
  if constexpr (CM == 2) {
    if (threadIdx.x < 256) s_tab[threadIdx.x] = otab[threadIdx.x];
    __syncthreads();
  }
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t s = g / (RS_C * H);
  const int u = (int)(g - s * (RS_C * H));
  const int h = u / RS_C, t = u % RS_C;
  const int64_t r = s * RS_C + t;
  const bool ok = r < nr;
  const int64_t row = ok ? (perm ? (int64_t)perm[r] : r) : 0;
  typename Epi::Pre pre{};
  if (ok && h == 0) pre = epi.pre(row);
  T sum = 0;
  if (ok) {
    const int64_t j0 = soff[s], nq = (soff[s + 1] - j0) / 4;
    const QuadCols qc = quad_setup<CM>(col, col16, sbase, code, coff, s_tab, s, j0, t, row);
    const T* vp = val + j0 * RS_C + t * 4;
#pragma unroll 2
    for (int64_t q = h; q < nq; q += H) sum += Quad<T>::dot(vp + q * (4 * RS_C), quad_cols<CM>(qc, q), x);
  }
  if (H >= 2) sum += __shfl_xor_sync(0xffffffffu, sum, 8);
  if (H >= 4) sum += __shfl_xor_sync(0xffffffffu, sum, 16);
  if (ok && h == 0) epi.post(row, sum, pre);
}

// threads the device keeps resident at once (SMs x 2048)
static int64_t device_threads() {
  static int64_t cached[64] = {0};
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int sms = 0, per = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaDeviceGetAttribute(&per, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    cached[dev] = (int64_t)sms * per;
  }
  return cached[dev];
}

template <class T, class Epi>
static void run_rows(Ctx& c, const RowsOp<T>& op, const T* x, const Epi& epi, const char* name = "csr_rows") {
  if (op.nr <= 0) return;
  // values and 4-byte columns, row pointers, x once, the epilogue's row vectors; stored form: the
  // columns as the layout holds them (4 bytes per entry, or 2 plus a 4-byte base per slice of 8
  // rows, or a one-byte code plus the 1 KB offset table)
  const double colb = op.c8 ? (double)op.nnz + 1024.0 : (op.c16 ? 2.0 * op.nnz + 0.5 * op.nr : 4.0 * op.nnz);
  const double rest = (double)op.nnz * sizeof(T) + 8.0 * (op.nr + 1) + (double)op.nc * sizeof(T) +
                      (double)op.nr * epi.row_bytes();
  ProfScope ps(c, name, rest + 4.0 * op.nnz, rest + colb);
  const int B = 256;
  if (op.sell) {
    // threads per row: enough for six waves of resident threads, at most 4
    const int64_t slices = (op.nr + RS_C - 1) / RS_C;
    int H = 1;
    // (each thread keeps at least two 4-slot groups of an average row)
    if (op.q == 4)
      while (H < 4 && op.nr * H < 6 * device_threads() && (double)op.nnz >= 8.0 * 2 * H * (double)op.nr) H *= 2;
    const int32_t* sc = op.scol.p;
    const uint16_t* sc16 = op.scol16.p;
    const int32_t* sb = op.sbase.p;
    const uint8_t* cd = op.scode.p;
    const int32_t* ot = op.otab.p;
    const int64_t* cf = op.coff.p;
    const unsigned g1 = grid_for(op.nr, B), g2 = grid_for(slices * RS_C * 2, B), g4 = grid_for(slices * RS_C * 4, B);
#define MGR_SELL_LAUNCH(CM)                                                                                       \
  do {                                                                                                           \
    if (H == 1)                                                                                                  \
      launch_pdl(c, k_rows_sell<T, Epi, 4, CM>, g1, B, 0, op.nr, op.soff.p, sc, sc16, sb, cd, cf, ot, op.sval.p,     \
                 op.perm.p, x, epi);                                                                             \
    else if (H == 2)                                                                                             \
      launch_pdl(c, k_rows_sell_split<T, Epi, 2, CM>, g2, B, 0, op.nr, op.soff.p, sc, sc16, sb, cd, cf, ot,          \
                 op.sval.p, op.perm.p, x, epi);                                                                  \
    else                                                                                                         \
      launch_pdl(c, k_rows_sell_split<T, Epi, 4, CM>, g4, B, 0, op.nr, op.soff.p, sc, sc16, sb, cd, cf, ot,          \
                 op.sval.p, op.perm.p, x, epi);                                                                  \
  } while (0)
    if (op.q == 4 && op.c8) MGR_SELL_LAUNCH(2);
    else if (op.q == 4 && op.c16) MGR_SELL_LAUNCH(1);
    else if (op.q == 4) MGR_SELL_LAUNCH(0);
    else
      launch_pdl(c, k_rows_sell<T, Epi, 1, 0>, g1, B, 0, op.nr, op.soff.p, sc, sc16, sb, cd, cf, ot, op.sval.p,
                 op.perm.p, x, epi);
#undef MGR_SELL_LAUNCH
    CU_LAUNCH();
    return;
  }
  const DCSR<T>& M = op.csr;
  double avg = M.nr ? (double)M.nnz / (double)M.nr : 0.0;
  // lanes per row: about four entries per lane or more
  if (avg <= 5.0) {
    launch_pdl(c, k_rows<T, 2, Epi>, grid_for(M.nr * 2, B), B, 0, M.nr, M.rp, M.ci, M.v, x, epi);
    CU_LAUNCH();
  } else if (avg <= 12.0) {
    launch_pdl(c, k_rows<T, 4, Epi>, grid_for(M.nr * 4, B), B, 0, M.nr, M.rp, M.ci, M.v, x, epi);
    CU_LAUNCH();
  } else if (avg <= 24.0) {
    launch_pdl(c, k_rows<T, 8, Epi>, grid_for(M.nr * 8, B), B, 0, M.nr, M.rp, M.ci, M.v, x, epi);
    CU_LAUNCH();
  } else if (avg <= 128.0) {
    launch_pdl(c, k_rows<T, 16, Epi>, grid_for(M.nr * 16, B), B, 0, M.nr, M.rp, M.ci, M.v, x, epi);
    CU_LAUNCH();
  } else {
    launch_pdl(c, k_rows<T, 32, Epi>, grid_for(M.nr * 32, B), B, 0, M.nr, M.rp, M.ci, M.v, x, epi);
    CU_LAUNCH();
  }
}

// Row epilogues: pre(row) loads what the epilogue needs before the row's product is formed, post(row,
// s, pre) finishes with the product s.
template <class T>
struct EpiFrelax {  // eFo[f] = eFi[f] + minv[f] (src_f - s)
  const int32_t* F; const T* src; const T* minv; const T* eFi; T* eFo;
  struct Pre { T b, m, e; };
  __device__ Pre pre(int64_t f) const { return {F ? src[F[f]] : src[f], minv[f], eFi[f]}; }
  __device__ void post(int64_t f, T s, const Pre& p) const { eFo[f] = p.e + p.m * (p.b - s); }
  double row_bytes() const { return (F ? 4 : 0) + 4.0 * sizeof(T); }
};
template <class T>
struct EpiRestrict {  // rnext[c] = base_c - s
  const int32_t* C; const T* r; T* rnext;
  struct Pre { T b; };
  __device__ Pre pre(int64_t c) const { return {C ? r[C[c]] : rnext[c]}; }
  __device__ void post(int64_t c, T s, const Pre& p) const { rnext[c] = p.b - s; }
  double row_bytes() const { return (C ? 4 : 0) + 2.0 * sizeof(T); }
};
template <class T>
struct EpiResid {
  const T* b; T* res;
  struct Pre { T b; };
  __device__ Pre pre(int64_t i) const { return {b[i]}; }
  __device__ void post(int64_t i, T s, const Pre& p) const { res[i] = p.b - s; }
  double row_bytes() const { return 2.0 * sizeof(T); }
};
template <class T>
struct EpiJacobi {
  const T* d; const T* b; const T* xi; T* xo;
  struct Pre { T d, b, x; };
  __device__ Pre pre(int64_t i) const { return {d[i], b[i], xi[i]}; }
  __device__ void post(int64_t i, T s, const Pre& p) const { xo[i] = p.x + p.d * (p.b - s); }
  double row_bytes() const { return 4.0 * sizeof(T); }
};
template <class T>
struct EpiStore {
  T* y;
  struct Pre {};
  __device__ Pre pre(int64_t) const { return {}; }
  __device__ void post(int64_t i, T s, const Pre&) const { y[i] = s; }
  double row_bytes() const { return 1.0 * sizeof(T); }
};
template <class T>
struct EpiAdd {
  T* y;
  struct Pre { T y; };
  __device__ Pre pre(int64_t i) const { return {y[i]}; }
  __device__ void post(int64_t i, T s, const Pre& p) const { y[i] = p.y + s; }
  double row_bytes() const { return 2.0 * sizeof(T); }
};

template <class T>
__global__ void k_frelax_first(int64_t nF, const int32_t* F, const T* src, const T* minv, T* eF) {
  pdl_wait();
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nF) return;
  eF[f] = minv[f] * (F ? src[F[f]] : src[f]);
}

template <class T>
void launch_frelax_first(Ctx& c, int64_t nF, const int32_t* F, const T* src, const T* minv, T* eF) {
  if (nF <= 0) return;
  launch_pdl(c, k_frelax_first<T>, grid_for(nF, 256), 256, 0, nF, F, src, minv, eF);
  CU_LAUNCH();
}
template <class T>
void launch_frelax_sweep(Ctx& c, const RowsOp<T>& Aff, const int32_t* F, const T* src, const T* minv, const T* eFi,
                         T* eFo, const char* name) {
  run_rows(c, Aff, eFi, EpiFrelax<T>{F, src, minv, eFi, eFo}, name);
}
template <class T>
void launch_restrict(Ctx& c, const RowsOp<T>& Acf, const int32_t* C, const T* r, const T* eF, T* rnext,
                     const char* name) {
  run_rows(c, Acf, eF, EpiRestrict<T>{C, r, rnext}, name);
}

// interpolation: C dofs take ec[c] (a scatter over the C list), F dofs eF[f] + W_p[f,:] ec (a
// vector-CSR pass over the rows of W_p); both add base[d] when given
template <class T, class TO>
__global__ void k_interp_c(int64_t nC, const int32_t* __restrict__ C, const T* __restrict__ ec,
                           const T* __restrict__ base, TO* __restrict__ out) {
  pdl_wait();
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nC) return;
  int32_t d = C[c];
  T v = ec[c];
  if (base) v += base[d];
  out[d] = (TO)v;
}
template <class T, class TO>
struct EpiInterpF {
  const int32_t* F; const T* eF; const T* base; TO* out;
  struct Pre { int32_t d; T e, b; };
  __device__ Pre pre(int64_t f) const {
    int32_t d = F[f];
    return {d, eF[f], base ? base[d] : T(0)};
  }
  __device__ void post(int64_t, T s, const Pre& p) const {
    T v = p.e + s;
    if (base) v += p.b;
    out[p.d] = (TO)v;
  }
  double row_bytes() const { return 4.0 + sizeof(T) + (base ? sizeof(T) : 0) + sizeof(TO); }
};

template <class T, class TO>
void launch_interp(Ctx& c, int64_t nF, const int32_t* F, int64_t nC, const int32_t* C, const RowsOp<T>& Wp,
                   const T* eF, const T* ec, const T* base, TO* out, const char* name) {
  if (nC > 0) {
    ProfScope ps(c, name, (double)nC * (4.0 + sizeof(T) + (base ? sizeof(T) : 0) + sizeof(TO)));
    launch_pdl(c, k_interp_c<T, TO>, grid_for(nC, 256), 256, 0, nC, C, ec, base, out);
    CU_LAUNCH();
  }
  if (nF > 0) run_rows(c, Wp, ec, EpiInterpF<T, TO>{F, eF, base, out}, name);
}

// dst[f] = src[idx[f]], and y += x
template <class T>
__global__ void k_gather(int64_t n, const int32_t* __restrict__ idx, const T* __restrict__ src, T* __restrict__ dst) {
  pdl_wait();
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f < n) dst[f] = src[idx[f]];
}
template <class T>
void launch_gather(Ctx& c, int64_t n, const int32_t* idx, const T* src, T* dst) {
  if (n <= 0) return;
  launch_pdl(c, k_gather<T>, grid_for(n, 256), 256, 0, n, idx, src, dst);
  CU_LAUNCH();
}
template <class T>
__global__ void k_axpy1(int64_t n, const T* __restrict__ x, T* __restrict__ y) {
  pdl_wait();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}
template <class T>
void launch_axpy(Ctx& c, int64_t n, const T* x, T* y) {
  if (n <= 0) return;
  launch_pdl(c, k_axpy1<T>, grid_for(n, 256), 256, 0, n, x, y);
  CU_LAUNCH();
}

// ---- the transposed preconditioner (M^-T) ------------------------------------------------------
template <class T>
struct EpiGatherAdd {  // out[c] = y[C[c]] + s   (P^T y = y_C + W_p^T y_F)
  const int32_t* C; const T* y; T* out;
  struct Pre { T y; };
  __device__ Pre pre(int64_t c) const { return {y[C[c]]}; }
  __device__ void post(int64_t c, T s, const Pre& p) const { out[c] = p.y + s; }
  double row_bytes() const { return 4.0 + 2.0 * sizeof(T); }
};
template <class T>
void launch_gather_add(Ctx& c, const RowsOp<T>& WpT, const int32_t* C, const T* y, T* out, const char* name) {
  run_rows(c, WpT, y, EpiGatherAdd<T>{C, y, out}, name);
}

// g[C[c]] = tc[c] for c < nC, g[F[f]] = gF[f] for f < nF
template <class T>
__global__ void k_scatter_cf(int64_t nC, const int32_t* C, const T* tc, int64_t nF, const int32_t* F, const T* gF,
                             T* g) {
  pdl_wait();
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nC) g[C[t]] = tc[t];
  else if (t < nC + nF) g[F[t - nC]] = gF[t - nC];
}
template <class T>
void launch_scatter_cf(Ctx& c, int64_t nC, const int32_t* C, const T* tc, int64_t nF, const int32_t* F, const T* gF,
                       T* g) {
  if (nC + nF <= 0) return;
  ProfScope ps(c, "scatter_cf", (double)(nC + nF) * (4.0 + 2.0 * sizeof(T)));
  launch_pdl(c, k_scatter_cf<T>, grid_for(nC + nF, 256), 256, 0, nC, C, tc, nF, F, gF, g);
  CU_LAUNCH();
}

// level-0 finish of M^-T with the global relaxation: z = g + B^T (y - A^T g), blocks of B^T given
template <class T>
struct EpiGRT {
  const double* y; const T* g; const T* bt; double* z;
  __device__ void operator()(int64_t I, T s0, T s1, T s2) const {
    T r0 = (T)y[3 * I] - s0, r1 = (T)y[3 * I + 1] - s1, r2 = (T)y[3 * I + 2] - s2;
    const T* b = bt + 9 * I;
    z[3 * I + 0] = (double)(g[3 * I + 0] + (b[0] * r0 + b[1] * r1 + b[2] * r2));
    z[3 * I + 1] = (double)(g[3 * I + 1] + (b[3] * r0 + b[4] * r1 + b[5] * r2));
    z[3 * I + 2] = (double)(g[3 * I + 2] + (b[6] * r0 + b[7] * r1 + b[8] * r2));
  }
};
template <class T>
void launch_bsr_grt(Ctx& c, const SellPattern& S, const T* valsT, const double* y, const T* g, const T* bt,
                    double* z) {
  ProfScope ps(c, "global_relax_t", (double)S.nnzb_real * (9 * sizeof(T) + 4) + 8.0 * (S.nb + 1) +
                                        (double)S.nb * (3 * sizeof(T) + 24 + 3 * sizeof(T) + 9 * sizeof(T) + 24));
  launch_bsr_sell<T, T>(c, S, valsT, g, EpiGRT<T>{y, g, bt, z});
}

template <class T>
__global__ void k_transpose_blocks(int64_t nb, const T* b, T* bt) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) bt[9 * I + 3 * p + q] = b[9 * I + 3 * q + p];
}
template <class T>
void launch_transpose_blocks(Ctx& c, int64_t nb, const T* b, T* bt) {
  if (nb <= 0) return;
  launch_pdl(c, k_transpose_blocks<T>, grid_for(nb, 256), 256, 0, nb, b, bt);
  CU_LAUNCH();
}

__global__ void k_dense_transpose(int64_t n, const double* a, double* at) {
  pdl_wait();
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int64_t i = t / n, j = t - i * n;
  at[j * n + i] = a[t];
}
void launch_dense_transpose(Ctx& c, int64_t n, const double* a, double* at) {
  if (n <= 0) return;
  launch_pdl(c, k_dense_transpose, grid_for(n * n, 256), 256, 0, n, a, at);
  CU_LAUNCH();
}

// columns j of a CSR matrix replaced by map[j]
__global__ void k_map_cols(int64_t nnz, int32_t* ci, const int32_t* map) {
  pdl_wait();
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nnz) ci[k] = map[ci[k]];
}
void launch_map_cols(Ctx& c, int64_t nnz, int32_t* ci, const int32_t* map) {
  if (nnz <= 0) return;
  launch_pdl(c, k_map_cols, grid_for(nnz, 256), 256, 0, nnz, ci, map);
  CU_LAUNCH();
}

template <class T>
__global__ void k_to_f64(int64_t n, const T* a, double* b) {
  pdl_wait();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
template <class T>
void launch_to_f64(Ctx& c, int64_t n, const T* a, double* b) {
  launch_pdl(c, k_to_f64<T>, grid_for(n, 256), 256, 0, n, a, b);
  CU_LAUNCH();
}

// ============================== AMG V-cycle pieces ==============================================
template <class T>
__global__ void k_scale_vec(int64_t n, const T* d, const T* b, T* x) {
  pdl_wait();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = d[i] * b[i];
}
template <class T>
void launch_scale(Ctx& c, int64_t n, const T* d, const T* b, T* x) {
  launch_pdl(c, k_scale_vec<T>, grid_for(n, 256), 256, 0, n, d, b, x);
  CU_LAUNCH();
}
template <class T>
void launch_resid(Ctx& c, const RowsOp<T>& A, const T* x, const T* b, T* res, const char* name) {
  run_rows(c, A, x, EpiResid<T>{b, res}, name);
}
template <class T>
void launch_jacobi(Ctx& c, const RowsOp<T>& A, const T* d, const T* b, const T* xi, T* xo, const char* name) {
  run_rows(c, A, xi, EpiJacobi<T>{d, b, xi, xo}, name);
}
template <class T>
void launch_spmv(Ctx& c, const RowsOp<T>& A, const T* x, T* y, const char* name) {
  run_rows(c, A, x, EpiStore<T>{y}, name);
}
template <class T>
void launch_prolong_add(Ctx& c, const RowsOp<T>& P, const T* xc, T* x, const char* name) {
  run_rows(c, P, xc, EpiAdd<T>{x}, name);
}

// x = inv b with the FP64 dense inverse of the coarsest operator: one warp per row
template <class T>
__global__ void k_dense_gemv(int64_t n, const double* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  pdl_wait();
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += inv[i * n + j] * (double)b[j];
  s = warp_sum(s);
  if (lane == 0) x[i] = (T)s;
}
template <class T>
void launch_dense_gemv(Ctx& c, int64_t n, const double* inv, const T* b, T* x) {
  if (n <= 0) return;
  launch_pdl(c, k_dense_gemv<T>, grid_for(n * 32, 256), 256, 0, n, inv, b, x);
  CU_LAUNCH();
}

__global__ void k_cast_f32(int64_t n, const double* a, float* b) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
void launch_cast_f32(Ctx& c, int64_t n, const double* a, float* b) {
  if (n <= 0) return;
  launch_pdl(c, k_cast_f32, grid_for(n, 256, 8192), 256, 0, n, a, b);
  CU_LAUNCH();
}

// ---- explicit instantiations -------------------------------------------------------------------
#define INST(T)                                                                                                    \
  template void launch_global_relax<T>(Ctx&, int64_t, const T*, const double*, T*);                               \
  template void launch_bsr_resid_split<T>(Ctx&, const SellPattern&, const T*, const double*, const T*,            \
                                          const int32_t*, T*, T*);                                                 \
  template void launch_frelax_first<T>(Ctx&, int64_t, const int32_t*, const T*, const T*, T*);                     \
  template void launch_frelax_sweep<T>(Ctx&, const RowsOp<T>&, const int32_t*, const T*, const T*, const T*, T*,   \
                                       const char*);                                                              \
  template void launch_restrict<T>(Ctx&, const RowsOp<T>&, const int32_t*, const T*, const T*, T*, const char*);  \
  template void launch_interp<T, T>(Ctx&, int64_t, const int32_t*, int64_t, const int32_t*, const RowsOp<T>&,     \
                                    const T*, const T*, const T*, T*, const char*);                                \
  template void launch_to_f64<T>(Ctx&, int64_t, const T*, double*);                                                \
  template void launch_scale<T>(Ctx&, int64_t, const T*, const T*, T*);                                            \
  template void launch_resid<T>(Ctx&, const RowsOp<T>&, const T*, const T*, T*, const char*);                     \
  template void launch_jacobi<T>(Ctx&, const RowsOp<T>&, const T*, const T*, const T*, T*, const char*);          \
  template void launch_spmv<T>(Ctx&, const RowsOp<T>&, const T*, T*, const char*);                                \
  template void launch_prolong_add<T>(Ctx&, const RowsOp<T>&, const T*, T*, const char*);                         \
  template void launch_gather_add<T>(Ctx&, const RowsOp<T>&, const int32_t*, const T*, T*, const char*);            \
  template void launch_scatter_cf<T>(Ctx&, int64_t, const int32_t*, const T*, int64_t, const int32_t*, const T*, T*);  \
  template void launch_bsr_grt<T>(Ctx&, const SellPattern&, const T*, const double*, const T*, const T*, double*);   \
  template void launch_transpose_blocks<T>(Ctx&, int64_t, const T*, T*);                                             \
  template void launch_gather<T>(Ctx&, int64_t, const int32_t*, const T*, T*);                                       \
  template void launch_axpy<T>(Ctx&, int64_t, const T*, T*);                                                         \
  template void launch_dense_gemv<T>(Ctx&, int64_t, const double*, const T*, T*);
INST(float)
INST(double)
#undef INST
template void launch_interp<float, double>(Ctx&, int64_t, const int32_t*, int64_t, const int32_t*,
                                           const RowsOp<float>&, const float*, const float*, const float*, double*,
                                           const char*);

}  // namespace mgr
