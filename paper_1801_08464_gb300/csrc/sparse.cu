// sparse.cu -- deterministic FP64 sparse setup primitives (compiled with --fmad=false).
//
// Every floating-point result here is produced by a fixed sequence of IEEE double operations
// (explicit __dmul_rn / __dadd_rn, no fused multiply-add, fixed summation order), so the products
// are reproducible bit for bit and independent of the launch configuration.
#include <climits>

#include "common.cuh"

namespace mgr {

// ---------------------------------------------------------------------------------------------
// BSR validation: rowptr starts at 0, ends at nnzb and is non-decreasing; columns in range and
// strictly ascending; each block row holds its diagonal block; markers in [0, MGR_MAX_LEVELS).
__global__ void k_bsr_validate(int64_t nb, int64_t nnzb, const int64_t* rp, const int32_t* ci, const int8_t* mk,
                               int* err) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  int64_t b = rp[I], e = rp[I + 1];
  bool ok = (b <= e) && (b >= 0) && (e <= nnzb);
  if (I == 0 && b != 0) ok = false;
  if (I == nb - 1 && e != nnzb) ok = false;
  bool diag = false;
  if (ok) {
    int32_t prev = -1;
    for (int64_t k = b; k < e; ++k) {
      int32_t j = ci[k];
      if (j < 0 || j >= nb || j <= prev) { ok = false; break; }
      if (j == I) diag = true;
      prev = j;
    }
  }
  if (mk)
    for (int p = 0; p < 3; ++p) {
      int8_t m = mk[3 * I + p];
      if (m < 0 || m >= MGR_MAX_LEVELS) ok = false;
    }
  if (!ok || !diag) atomicOr(err, EBIT_PATTERN);
}

void bsr3_validate_launch(Ctx& c, const mgr_bsr3_t& A, const int8_t* marker) {
  if (A.nb <= 0 || A.nnzb < A.nb || !A.rowptr || !A.colind || !A.values)
    throw Error(MGR_ERR_INVALID_ARG, "bsr3: bad sizes or null pointers");
  if (A.nb >= (1ll << 31) / 3) throw Error(MGR_ERR_UNSUPPORTED, "bsr3: 3*nb must fit in int32");
  k_bsr_validate<<<grid_for(A.nb, 256), 256, 0, c.s>>>(A.nb, A.nnzb, A.rowptr, A.colind, marker, c.d_err);
  CU_LAUNCH();
}
void bsr3_validate(Ctx& c, const mgr_bsr3_t& A, const int8_t* marker) {
  bsr3_validate_launch(c, A, marker);
  check_errors(c, "bsr3_validate");
}

// ---------------------------------------------------------------------------------------------
// Scalar CSR view of the BSR matrix with exact zeros dropped: row 3I+p collects, over the blocks
// of block row I in ascending column order and q = 0..2, the nonzero entries (3J+q, B[p][q]).
__global__ void k_bsr_csr_count(int64_t nb, const int64_t* rp, const double* v, int64_t* cnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= 3 * nb) return;
  int64_t I = r / 3;
  int p = (int)(r - 3 * I);
  int64_t s = 0;
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k)
    for (int q = 0; q < 3; ++q) s += (v[9 * k + 3 * p + q] != 0.0);
  cnt[r] = s;
}
// a group of RG lanes per scalar row: entry t of row 3I+p is value q = t % 3 of block b0 + t / 3
__global__ void __launch_bounds__(256) k_bsr_csr_fill(int64_t nb, const int64_t* rp, const int32_t* ci,
                                                      const double* v, const int64_t* orp, int32_t* oci, double* ov) {
  const RowGroup G = row_group();
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / RG;
  const bool act = r < 3 * nb;
  int64_t b0 = 0, o = 0;
  int p = 0, len = 0;
  if (act) {
    const int64_t I = r / 3;
    p = (int)(r - 3 * I);
    b0 = rp[I];
    len = 3 * (int)(rp[I + 1] - b0);
    o = orp[r];
  }
  const int rounds = warp_max_int((len + RG - 1) / RG);
  for (int rd = 0; rd < rounds; ++rd) {
    const int t = rd * RG + G.g;
    const bool in = act && t < len;
    double x = 0.0;
    int64_t k = 0;
    int q = 0;
    if (in) {
      k = b0 + t / 3;
      q = t - 3 * (t / 3);
      x = v[9 * k + 3 * p + q];
    }
    const bool nz = in && x != 0.0;
    const unsigned bn = __ballot_sync(0xffffffffu, nz) & G.gmask;
    if (nz) {
      const int64_t d = o + __popc(bn & G.below);
      oci[d] = 3 * ci[k] + q;
      ov[d] = x;
    }
    o += __popc(bn);
  }
}

void bsr3_to_csr(Ctx& c, const mgr_bsr3_t& A, DCSR<double>& out) {
  int64_t n = 3 * A.nb;
  DBuf<int64_t> cnt(c, n);
  out.nr = out.nc = n;
  out.rp.alloc(c, n + 1);
  k_bsr_csr_count<<<grid_for(n, 256), 256, 0, c.s>>>(A.nb, A.rowptr, A.values, cnt.p);
  CU_LAUNCH();
  out.nnz = counts_to_rowptr(c, cnt.p, out.rp.p, n);
  out.ci.alloc(c, out.nnz);
  out.v.alloc(c, out.nnz);
  k_bsr_csr_fill<<<grid_for(n * RG, 256), 256, 0, c.s>>>(A.nb, A.rowptr, A.colind, A.values, out.rp.p, out.ci.p,
                                                         out.v.p);
  CU_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// Inverse of each 3x3 diagonal block by the adjugate over the determinant (cofactor expansion
// along row 0); a zero or non-finite determinant sets EBIT_SINGULAR.
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

__global__ void k_block_inverse(int64_t nb, const int64_t* rp, const int32_t* ci, const double* v, double* binv, int* err) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  int64_t k = find_i32(ci, rp[I], rp[I + 1], (int32_t)I);
  double* r = binv + 9 * I;
  if (k < 0) { atomicOr(err, EBIT_PATTERN); return; }
  const double* b = v + 9 * k;
  double c00 = ds(dm(b[4], b[8]), dm(b[5], b[7]));
  double c01 = ds(dm(b[5], b[6]), dm(b[3], b[8]));
  double c02 = ds(dm(b[3], b[7]), dm(b[4], b[6]));
  double det = dd(dd(dm(b[0], c00), dm(b[1], c01)), dm(b[2], c02));
  if (det == 0.0 || !isfinite(det)) {
    atomicOr(err, EBIT_SINGULAR);
    for (int t = 0; t < 9; ++t) r[t] = 0.0;
    return;
  }
  double id = __ddiv_rn(1.0, det);
  r[0] = dm(c00, id);
  r[1] = dm(ds(dm(b[2], b[7]), dm(b[1], b[8])), id);
  r[2] = dm(ds(dm(b[1], b[5]), dm(b[2], b[4])), id);
  r[3] = dm(c01, id);
  r[4] = dm(ds(dm(b[0], b[8]), dm(b[2], b[6])), id);
  r[5] = dm(ds(dm(b[2], b[3]), dm(b[0], b[5])), id);
  r[6] = dm(c02, id);
  r[7] = dm(ds(dm(b[1], b[6]), dm(b[0], b[7])), id);
  r[8] = dm(ds(dm(b[0], b[4]), dm(b[1], b[3])), id);
}

void bsr3_block_inverse(Ctx& c, const mgr_bsr3_t& A, double* binv) {
  k_block_inverse<<<grid_for(A.nb, 128), 128, 0, c.s>>>(A.nb, A.rowptr, A.colind, A.values, binv, c.d_err);
  CU_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// Sorting helpers (bitonic networks in shared memory).
__device__ __forceinline__ void block_bitonic_keys(int32_t* key, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int x = t ^ j;
        if (x > t) {
          bool up = (t & k) == 0;
          int32_t a = key[t], b = key[x];
          if ((a > b) == up) { key[t] = b; key[x] = a; }
        }
      }
      __syncthreads();
    }
}
__device__ __forceinline__ int next_pow2(int x) {
  int n = 1;
  while (n < x) n <<= 1;
  return n;
}

// ---------------------------------------------------------------------------------------------
// SpGEMM.  Rows with at most FUSE_CAP products (ub_i = sum of the B row lengths selected by row i of
// A) are formed in one pass by the fused kernels below.  Longer rows take a symbolic pass (the
// sorted union of the selected B rows' columns: a block with a shared hash table for
// ub <= SYM_BCAP, a block with a bitmap over the columns of C for nc <= SYM_BITS, else a bounded
// 32K-slot hash) and a numeric pass.
constexpr int FUSE_CAP = 2048;  // rows with up to FUSE_CAP products take the fused (one-pass) kernels
constexpr int64_t SPGEMM_STAGE = 128ll << 20;  // staged products per batch of fused rows
constexpr int SYM_BCAP = 8192;
constexpr int SYM_BHASH = 16384;
constexpr int64_t SYM_BITS = 1 << 20;

__global__ void k_spgemm_ub(int64_t m, const int64_t* arp, const int32_t* aci, const int64_t* brp, int64_t* ub,
                            int* n_mid, int32_t* mid, int* n_big, int32_t* big) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t s = 0;
  for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
    int32_t k = aci[p];
    s += brp[k + 1] - brp[k];
  }
  ub[i] = s;
  if (s > SYM_BCAP) big[atomicAdd(n_big, 1)] = (int32_t)i;
  else if (s > FUSE_CAP) mid[atomicAdd(n_mid, 1)] = (int32_t)i;
}

__device__ __forceinline__ uint32_t hash32(int32_t k) { return (uint32_t)k * 2654435761u; }

template <int MODE>
__global__ void k_sym_block(const int32_t* rows, const int64_t* arp, const int32_t* aci, const int64_t* brp,
                            const int32_t* bci, int64_t* cnt, const int64_t* crp, int32_t* cci) {
  extern __shared__ int32_t smem[];
  int32_t* T = smem;               // SYM_BHASH
  int32_t* K = smem + SYM_BHASH;   // SYM_BCAP
  __shared__ int ucount;
  int64_t i = rows[blockIdx.x];
  for (int t = threadIdx.x; t < SYM_BHASH; t += blockDim.x) T[t] = -1;
  if (threadIdx.x == 0) ucount = 0;
  __syncthreads();
  int64_t a0 = arp[i], a1 = arp[i + 1];
  // warp w takes the A entries w, w + nwarps, ...; its lanes insert the selected B row (set union:
  // order irrelevant), so short B rows still keep most lanes busy
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int64_t p = a0 + (threadIdx.x >> 5); p < a1; p += nwarp) {
    int32_t k = aci[p];
    for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
      int32_t key = bci[q];
      uint32_t h = hash32(key) & (SYM_BHASH - 1);
      while (true) {
        int32_t prev = atomicCAS(&T[h], -1, key);
        if (prev == -1) { atomicAdd(&ucount, 1); break; }
        if (prev == key) break;
        h = (h + 1) & (SYM_BHASH - 1);
      }
    }
  }
  __syncthreads();
  int u = ucount;
  if (MODE == 0) {
    if (threadIdx.x == 0) cnt[i] = u;
    return;
  }
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  // compaction (order irrelevant: sorted afterwards)
  for (int t = threadIdx.x; t < SYM_BHASH; t += blockDim.x) {
    int32_t key = T[t];
    if (key >= 0) K[atomicAdd(&base, 1)] = key;
  }
  __syncthreads();
  int n2 = next_pow2(u);
  for (int t = u + threadIdx.x; t < n2; t += blockDim.x) K[t] = INT_MAX;
  __syncthreads();
  block_bitonic_keys(K, n2);
  int64_t o = crp[i];
  for (int t = threadIdx.x; t < u; t += blockDim.x) cci[o + t] = K[t];
}

// Rows with more than SYM_BCAP products when C has more than SYM_BITS columns: a block-wide hash of
// SYM_GHASH slots holding at most SYM_GCAP distinct columns (a row with more sets EBIT_CAPACITY and
// is left empty).  Probing is bounded by the table size, so a full table ends the insertion.
constexpr int SYM_GHASH = 32768;
constexpr int SYM_GCAP = 16384;

template <int MODE>
__global__ void __launch_bounds__(1024) k_sym_bighash(const int32_t* rows, const int64_t* arp, const int32_t* aci,
                                                      const int64_t* brp, const int32_t* bci, int64_t* cnt,
                                                      const int64_t* crp, int32_t* cci, int* err) {
  extern __shared__ int32_t smem[];
  int32_t* T = smem;               // SYM_GHASH
  int32_t* K = smem + SYM_GHASH;   // SYM_GCAP
  __shared__ int ucount, full;
  int64_t i = rows[blockIdx.x];
  for (int t = threadIdx.x; t < SYM_GHASH; t += blockDim.x) T[t] = -1;
  if (threadIdx.x == 0) { ucount = 0; full = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int64_t p = arp[i] + (threadIdx.x >> 5); p < arp[i + 1]; p += nwarp) {
    int32_t k = aci[p];
    for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
      int32_t key = bci[q];
      uint32_t h = hash32(key) & (SYM_GHASH - 1);
      int probes = 0;
      while (true) {
        int32_t prev = atomicCAS(&T[h], -1, key);
        if (prev == -1) { atomicAdd(&ucount, 1); break; }
        if (prev == key) break;
        h = (h + 1) & (SYM_GHASH - 1);
        if (++probes >= SYM_GHASH) { full = 1; break; }
      }
    }
  }
  __syncthreads();
  int u = ucount;
  if (full || u > SYM_GCAP) {
    if (threadIdx.x == 0) {
      atomicOr(err, EBIT_CAPACITY);
      if (MODE == 0) cnt[i] = 0;
    }
    return;
  }
  if (MODE == 0) {
    if (threadIdx.x == 0) cnt[i] = u;
    return;
  }
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < SYM_GHASH; t += blockDim.x) {
    int32_t key = T[t];
    if (key >= 0) K[atomicAdd(&base, 1)] = key;
  }
  __syncthreads();
  int n2 = next_pow2(u);
  for (int t = u + threadIdx.x; t < n2; t += blockDim.x) K[t] = INT_MAX;
  __syncthreads();
  block_bitonic_keys(K, n2);
  int64_t o = crp[i];
  for (int t = threadIdx.x; t < u; t += blockDim.x) cci[o + t] = K[t];
}

// bitmap over the columns [0, nc), nc <= SYM_BITS; 1024 threads, each owning consecutive words
template <int MODE>
__global__ void __launch_bounds__(1024) k_sym_bitmap(const int32_t* rows, int64_t nc, const int64_t* arp,
                                                     const int32_t* aci, const int64_t* brp, const int32_t* bci,
                                                     int64_t* cnt, const int64_t* crp, int32_t* cci) {
  extern __shared__ uint32_t bits[];
  __shared__ int wsum[32];
  int nw = (int)((nc + 31) >> 5);
  int64_t i = rows[blockIdx.x];
  for (int t = threadIdx.x; t < nw; t += blockDim.x) bits[t] = 0u;
  __syncthreads();
  {
    const int ln = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int64_t p = arp[i] + (threadIdx.x >> 5); p < arp[i + 1]; p += nwarp) {
      int32_t k = aci[p];
      for (int64_t q = brp[k] + ln; q < brp[k + 1]; q += 32) {
        int32_t key = bci[q];
        atomicOr(&bits[key >> 5], 1u << (key & 31));
      }
    }
  }
  __syncthreads();
  int per = (nw + blockDim.x - 1) / blockDim.x;
  int w0 = threadIdx.x * per;
  int s = 0;
  for (int t = 0; t < per; ++t)
    if (w0 + t < nw) s += __popc(bits[w0 + t]);
  // block exclusive scan of s
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = s;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int y = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    wsum[lane] = y;
  }
  __syncthreads();
  int before = (wid ? wsum[wid - 1] : 0) + x - s;
  if (MODE == 0) {
    if (threadIdx.x == blockDim.x - 1) cnt[i] = before + s;
    return;
  }
  int64_t o = crp[i] + before;
  for (int t = 0; t < per; ++t) {
    int wi = w0 + t;
    if (wi >= nw) break;
    uint32_t b = bits[wi];
    while (b) {
      int bit = __ffs(b) - 1;
      cci[o++] = (wi << 5) + bit;
      b &= b - 1;
    }
  }
}

// Symbolic pass for the rows with more than FUSE_CAP products: count (mode 0) or write the sorted
// distinct columns (mode 1) of the listed rows.
static void sym_pass(Ctx& c, int mode, const DCSR<double>& A, const DCSR<double>& B, const int32_t* mid, int nmid,
                     const int32_t* big, int nbig, int64_t* cnt, DCSR<double>& C) {
  ProfScope ps(c, mode == 0 ? "sym_count" : "sym_fill");
  if (nmid > 0) {
    ProfScope ps2(c, "sym_block");
    size_t sh = sizeof(int32_t) * (SYM_BHASH + SYM_BCAP);
    if (mode == 0) {
      CU(cudaFuncSetAttribute(k_sym_block<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_block<0><<<nmid, 512, sh, c.s>>>(mid, A.rp, A.ci, B.rp, B.ci, cnt, nullptr, nullptr);
      CU_LAUNCH();
    } else {
      CU(cudaFuncSetAttribute(k_sym_block<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_block<1><<<nmid, 512, sh, c.s>>>(mid, A.rp, A.ci, B.rp, B.ci, nullptr, C.rp, C.ci);
      CU_LAUNCH();
    }
  }
  if (nbig > 0 && B.nc <= SYM_BITS) {
    ProfScope ps3(c, "sym_bitmap");
    size_t sh = sizeof(uint32_t) * (size_t)((B.nc + 31) / 32);
    if (mode == 0) {
      CU(cudaFuncSetAttribute(k_sym_bitmap<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_bitmap<0><<<nbig, 1024, sh, c.s>>>(big, B.nc, A.rp, A.ci, B.rp, B.ci, cnt, nullptr, nullptr);
      CU_LAUNCH();
    } else {
      CU(cudaFuncSetAttribute(k_sym_bitmap<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_bitmap<1><<<nbig, 1024, sh, c.s>>>(big, B.nc, A.rp, A.ci, B.rp, B.ci, nullptr, C.rp, C.ci);
      CU_LAUNCH();
    }
  } else if (nbig > 0) {
    ProfScope ps3(c, "sym_bitmap");
    size_t sh = sizeof(int32_t) * (SYM_GHASH + SYM_GCAP);
    if (mode == 0) {
      CU(cudaFuncSetAttribute(k_sym_bighash<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_bighash<0><<<nbig, 1024, sh, c.s>>>(big, A.rp, A.ci, B.rp, B.ci, cnt, nullptr, nullptr, c.d_err);
      CU_LAUNCH();
      check_errors(c, "spgemm: long rows");
    } else {
      CU(cudaFuncSetAttribute(k_sym_bighash<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
      k_sym_bighash<1><<<nbig, 1024, sh, c.s>>>(big, A.rp, A.ci, B.rp, B.ci, nullptr, C.rp, C.ci, c.d_err);
      CU_LAUNCH();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// SpGEMM numeric.  Every entry of C is the sum over ascending intermediate index k of a_ik b_kj,
// starting from 0.0 (Gustavson's order), computed with explicit round-to-nearest multiplies and adds.
//
// k_spgemm_numeric_expand (rows with at most NX_CAPA entries in A and NX_CAPC in C): a warp per row
// enumerates the products of row i in (k, q) order, 32 at a time, one per lane.  Lanes whose products
// land on the same output entry are grouped with __match_any_sync; the lowest lane of a group adds the
// group's products in lane order, and groups of successive chunks are added in chunk order, so each
// entry still receives its products in ascending k.  All lanes work even when the rows of B are short.
// k_spgemm_numeric (the remaining rows): the A row is walked in ascending order; for each k the lanes
// add a_ik b_kj to entry j of the sorted C row found by binary search (distinct j within one B row,
// __syncwarp between successive k), accumulating in the output array.
constexpr int NUM_WARPS = 8;
constexpr int NX_WARPS = 4;
constexpr int NX_CAPA = 256;
constexpr int NX_CAPC = 512;

__global__ void __launch_bounds__(32 * NX_WARPS) k_spgemm_numeric_expand(
    int64_t m, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, const double* __restrict__ av,
    const int64_t* __restrict__ brp, const int32_t* __restrict__ bci, const double* __restrict__ bv,
    const int64_t* __restrict__ crp, const int32_t* __restrict__ cci, double* __restrict__ cv,
    const int64_t* __restrict__ ub) {
  __shared__ int32_t scol[NX_WARPS][NX_CAPC];
  __shared__ double sacc[NX_WARPS][NX_CAPC];
  __shared__ int32_t sstart[NX_WARPS][NX_CAPA + 1];
  __shared__ int64_t sbeg[NX_WARPS][NX_CAPA];
  __shared__ double sa[NX_WARPS][NX_CAPA];
  __shared__ double sval[NX_WARPS][32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * NX_WARPS + w;
  if (i >= m) return;
  if (ub[i] <= FUSE_CAP) return;  // done by the fused kernel
  int64_t a0 = arp[i], c0 = crp[i];
  int na = (int)(arp[i + 1] - a0), L = (int)(crp[i + 1] - c0);
  if (na > NX_CAPA || L > NX_CAPC) return;  // handled by k_spgemm_numeric
  for (int t = lane; t < L; t += 32) { scol[w][t] = cci[c0 + t]; sacc[w][t] = 0.0; }
  // exclusive scan of the B row lengths along the A row
  int carry = 0;
  for (int p0 = 0; p0 < na; p0 += 32) {
    int p = p0 + lane;
    int len = 0;
    if (p < na) {
      int32_t k = aci[a0 + p];
      int64_t b0 = brp[k];
      len = (int)(brp[k + 1] - b0);
      sbeg[w][p] = b0;
      sa[w][p] = av[a0 + p];
    }
    int x = len;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (p < na) sstart[w][p] = carry + x - len;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) sstart[w][na] = carry;
  __syncwarp();
  int P = carry;
  for (int t0 = 0; t0 < P; t0 += 32) {
    int t = t0 + lane;
    int pos = -1 - lane;  // distinct sentinel: idle lanes never group with each other
    double val = 0.0;
    if (t < P) {
      // product t belongs to A entry p with sstart[p] <= t < sstart[p+1]
      int lo = 0, hi = na;
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (sstart[w][mid] <= t) lo = mid; else hi = mid;
      }
      int64_t q = sbeg[w][lo] + (t - sstart[w][lo]);
      val = __dmul_rn(sa[w][lo], bv[q]);
      pos = (int)lower_bound_i32(scol[w], 0, L, bci[q]);
    }
    unsigned grp = __match_any_sync(0xffffffffu, pos);
    sval[w][lane] = val;
    __syncwarp();
    if (t < P && lane == __ffs(grp) - 1) {
      double acc = sacc[w][pos];
      unsigned g = grp;
      while (g) {
        int l = __ffs(g) - 1;
        acc = __dadd_rn(acc, sval[w][l]);
        g &= g - 1;
      }
      sacc[w][pos] = acc;
    }
    __syncwarp();
  }
  for (int t = lane; t < L; t += 32) cv[c0 + t] = sacc[w][t];
}

__global__ void __launch_bounds__(32 * NUM_WARPS) k_spgemm_numeric(int64_t m, const int64_t* arp, const int32_t* aci,
                                                                    const double* av, const int64_t* brp,
                                                                    const int32_t* bci, const double* bv,
                                                                    const int64_t* crp, const int32_t* cci, double* cv,
                                                                    const int64_t* ub) {
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * NUM_WARPS + w;
  if (i >= m || ub[i] <= FUSE_CAP) return;
  int64_t c0 = crp[i], c1 = crp[i + 1];
  int64_t L = c1 - c0;
  if (arp[i + 1] - arp[i] <= NX_CAPA && L <= NX_CAPC) return;  // done by the expand kernel
  const int32_t* col = cci + c0;
  double* acc = cv + c0;
  for (int64_t t = lane; t < L; t += 32) acc[t] = 0.0;
  __syncwarp();
  for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
    int32_t k = aci[p];
    double a = av[p];
    for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
      int64_t pos = lower_bound_i32(col, 0, L, bci[q]);
      acc[pos] = __dadd_rn(acc[pos], __dmul_rn(a, bv[q]));
    }
    __syncwarp();
  }
}

// Stores the u distinct (column, value) pairs K[0..u), V[0..u) (any order, u <= 128) at
// ocol/oval in ascending column order: each lane holds up to 4 pairs and counts, in one pass over the
// keys (broadcast shared-memory reads), how many are smaller; that count is the pair's position.
template <int NH>
__device__ __forceinline__ void warp_rank_store(const int32_t* K, const double* V, int u, int lane, int32_t* ocol,
                                                double* oval) {
  int32_t key[NH];
  int r[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    int t = lane + 32 * h;
    key[h] = t < u ? K[t] : INT_MAX;
    r[h] = 0;
  }
  // the rank of a key is the number of smaller keys; four keys per (broadcast) 16-byte read
  int j = 0;
  for (; j + 4 <= u; j += 4) {
    const int4 kk = *reinterpret_cast<const int4*>(K + j);
#pragma unroll
    for (int h = 0; h < NH; ++h)
      r[h] += (kk.x < key[h]) + (kk.y < key[h]) + (kk.z < key[h]) + (kk.w < key[h]);
  }
  for (; j < u; ++j) {
    const int32_t kj = K[j];
#pragma unroll
    for (int h = 0; h < NH; ++h) r[h] += (kj < key[h]);
  }
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    int t = lane + 32 * h;
    if (t < u) { ocol[r[h]] = key[h]; oval[r[h]] = V[t]; }
  }
}

// Places the u <= 128 distinct (column, value) pairs of K / V at their ranks in ocol / oval (sorted
// by column): each lane ranks up to four keys against all u keys.
__device__ __forceinline__ void warp_rank_store128(const int32_t* K, const double* V, int u, int lane,
                                                   int32_t* ocol, double* oval) {
  if (u <= 32) warp_rank_store<1>(K, V, u, lane, ocol, oval);
  else if (u <= 64) warp_rank_store<2>(K, V, u, lane, ocol, oval);
  else if (u <= 96) warp_rank_store<3>(K, V, u, lane, ocol, oval);
  else warp_rank_store<4>(K, V, u, lane, ocol, oval);
}

// Fused product for rows with at most TT_CAP products, one thread per row: the products are taken
// in (k, q) order and merged into a short sorted list in shared memory (a new column is inserted
// with 0.0 + its product, a repeated column adds its product), so every entry is summed from 0.0 in
// ascending k exactly as in the warp kernels, with no hashing and no sort pass.
constexpr int TT_CAP = 32;
constexpr int TT_THREADS = 64;

__global__ void __launch_bounds__(TT_THREADS) k_spgemm_tiny(
    int64_t r0, int64_t r1, int64_t sbase, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
    const double* __restrict__ av, const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
    const double* __restrict__ bv, const int64_t* __restrict__ ub, const int64_t* __restrict__ soff,
    int32_t* __restrict__ scol, double* __restrict__ sval, int64_t* __restrict__ cnt) {
  __shared__ int32_t sc[TT_CAP][TT_THREADS];
  __shared__ double sv[TT_CAP][TT_THREADS];
  const int t = threadIdx.x;
  const int64_t i = r0 + (int64_t)blockIdx.x * TT_THREADS + t;
  if (i >= r1) return;
  if (ub[i] > TT_CAP) return;
  int u = 0;
  for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
    const int32_t k = aci[p];
    const double a = av[p];
    for (int64_t q = brp[k]; q < brp[k + 1]; ++q) {
      const int32_t j = bci[q];
      const double prod = __dmul_rn(a, bv[q]);
      int pos = u;
      while (pos > 0 && sc[pos - 1][t] > j) --pos;
      if (pos > 0 && sc[pos - 1][t] == j) {
        sv[pos - 1][t] = __dadd_rn(sv[pos - 1][t], prod);
      } else {
        for (int e = u; e > pos; --e) { sc[e][t] = sc[e - 1][t]; sv[e][t] = sv[e - 1][t]; }
        sc[pos][t] = j;
        sv[pos][t] = __dadd_rn(0.0, prod);
        ++u;
      }
    }
  }
  const int64_t o = soff[i] - sbase;
  for (int e = 0; e < u; ++e) { scol[o + e] = sc[e][t]; sval[o + e] = sv[e][t]; }
  cnt[i] = u;
}

// Fused product of one row (a warp), the common case of the setup products: products are taken 32
// at a time in (k, q) order, i.e. ascending intermediate index k (lane t holds product t0 + t; its A
// entry comes from a scan of the B row lengths kept in shared memory, and the next chunk's loads are
// issued before the current chunk is added).  The A row is taken in batches of CAPA entries (the
// scan's capacity), in order.  Lanes holding the same column form a group (__match_any_sync); the
// group's lowest lane adds the group's products in lane order to the column's running sum in a
// row-sized shared hash table.  Every sum therefore starts at 0.0 and adds its products in ascending
// k (Gustavson's order).  Only the distinct columns are then sorted (rank placement up to 128, else
// bitonic, sums carried) and staged at scol/sval + o.
struct ChunkSmem {
  int32_t* K;     // [slots] hash keys
  double* V;      // [slots] running sums
  int32_t* sst;   // [capa + 1] product offsets of the batch's A entries
  int64_t* sbg;   // [capa] B row starts
  double* sa;     // [capa] A values
  double* gv;     // [32] the chunk's products
};

// Table size: a power of two of at least 2 U (load at most one half).  CLEAN: the table is all
// free at entry and is left all free (the compaction scan frees each slot it reads), so a warp
// walking many rows initialises it once.
__device__ __forceinline__ int chunk_table_size(int U) {
  int H = 32;
  while (H < 2 * U) H <<= 1;
  return H;
}

template <int SLOTS, int CAPA, bool CLEAN, int LIMIT>
__device__ __forceinline__ bool chunk_row(int64_t i, int U, const int64_t* __restrict__ arp,
                                          const int32_t* __restrict__ aci, const double* __restrict__ av,
                                          const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                          const double* __restrict__ bv, int64_t o, int32_t* __restrict__ scol,
                                          double* __restrict__ sval, int64_t* __restrict__ cnt, const ChunkSmem& sm) {
  const int lane = threadIdx.x & 31;
  int32_t* K = sm.K;
  double* Vv = sm.V;
  const int H = chunk_table_size(U) < SLOTS ? chunk_table_size(U) : SLOTS;
  int distinct = 0;  // keys in the table (a table of SLOTS slots stops the row at LIMIT keys)
  if (!CLEAN)
    for (int t = lane; t < H; t += 32) { K[t] = -1; Vv[t] = 0.0; }
  const int64_t a0 = arp[i], a1 = arp[i + 1];
  for (int64_t pb = a0; pb < a1; pb += CAPA) {
    const int na = (int)((a1 - pb) < CAPA ? (a1 - pb) : CAPA);
    __syncwarp();
    int carry = 0;
    for (int p0 = 0; p0 < na; p0 += 32) {
      int p = p0 + lane;
      int len = 0;
      if (p < na) {
        int32_t k = aci[pb + p];
        int64_t b0 = brp[k];
        len = (int)(brp[k + 1] - b0);
        sm.sbg[p] = b0;
        sm.sa[p] = av[pb + p];
      }
      int x = len;
      for (int of = 1; of < 32; of <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, of);
        if (lane >= of) x += y;
      }
      if (p < na) sm.sst[p] = carry + x - len;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) sm.sst[na] = carry;
    __syncwarp();
    const int Ub = carry;
    // product t of the batch -> (column, value)
    auto fetch = [&](int t, int32_t& col, double& val) {
      col = -1 - lane;
      val = 0.0;
      if (t < Ub) {
        int lo = 0, hi = na;
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (sm.sst[mid] <= t) lo = mid; else hi = mid;
        }
        int64_t q = sm.sbg[lo] + (t - sm.sst[lo]);
        col = bci[q];
        val = __dmul_rn(sm.sa[lo], bv[q]);
      }
    };
    int32_t ncol;
    double nval;
    fetch(lane, ncol, nval);
    for (int t0 = 0; t0 < Ub; t0 += 32) {
      int32_t col = ncol;
      double val = nval;
      if (t0 + 32 < Ub) fetch(t0 + 32 + lane, ncol, nval);
      unsigned grp = __match_any_sync(0xffffffffu, col);
      sm.gv[lane] = val;
      __syncwarp();
      bool fresh = false;
      if (col >= 0 && lane == __ffs(grp) - 1) {
        uint32_t h = hash32(col) & (H - 1);
        while (true) {
          int32_t prev = atomicCAS(&K[h], -1, col);
          if (prev == -1 || prev == col) { fresh = prev == -1; break; }
          h = (h + 1) & (H - 1);
        }
        double acc = Vv[h];
        unsigned g = grp;
        while (g) {
          int l = __ffs(g) - 1;
          acc = __dadd_rn(acc, sm.gv[l]);
          g &= g - 1;
        }
        Vv[h] = acc;
      }
      distinct += __popc(__ballot_sync(0xffffffffu, fresh));
      __syncwarp();
      if (distinct > LIMIT) {  // the row needs a larger table
        if (CLEAN) {
          for (int t = lane; t < H; t += 32) { K[t] = -1; Vv[t] = 0.0; }
          __syncwarp();
        }
        return false;
      }
    }
  }
  __syncwarp();
  // compact the occupied slots, sort them by column, stage
  int base = 0;
  for (int t0 = 0; t0 < H; t0 += 32) {
    int t = t0 + lane;
    int32_t key = t < H ? K[t] : -1;
    double v = t < H ? Vv[t] : 0.0;
    unsigned msk = __ballot_sync(0xffffffffu, key >= 0);
    __syncwarp();
    if (CLEAN && t < H) { K[t] = -1; Vv[t] = 0.0; }
    __syncwarp();
    if (key >= 0) {
      int pos = base + __popc(msk & ((1u << lane) - 1));
      K[pos] = key;
      Vv[pos] = v;
    }
    base += __popc(msk);
    __syncwarp();
  }
  const int u = base;
  if (u <= 128) {
    warp_rank_store128(K, Vv, u, lane, scol + o, sval + o);
    if (lane == 0) cnt[i] = u;
    __syncwarp();
    if (CLEAN) {
      for (int t = lane; t < u; t += 32) { K[t] = -1; Vv[t] = 0.0; }
      __syncwarp();
    }
    return true;
  }
  int n2 = 1;
  while (n2 < u) n2 <<= 1;
  for (int t = u + lane; t < n2; t += 32) K[t] = INT_MAX;
  __syncwarp();
  for (int k2 = 2; k2 <= n2; k2 <<= 1)
    for (int j = k2 >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < n2; t += 32) {
        int x = t ^ j;
        if (x > t) {
          bool up = (t & k2) == 0;
          int32_t ka = K[t], kb = K[x];
          if ((ka > kb) == up) {
            K[t] = kb; K[x] = ka;
            double va = Vv[t]; Vv[t] = Vv[x]; Vv[x] = va;
          }
        }
      }
      __syncwarp();
    }
  for (int t = lane; t < u; t += 32) { scol[o + t] = K[t]; sval[o + t] = Vv[t]; }
  if (lane == 0) cnt[i] = u;
  __syncwarp();
  if (CLEAN) {
    for (int t = lane; t < n2; t += 32) { K[t] = -1; Vv[t] = 0.0; }
    __syncwarp();
  }
  return true;
}

// Rows of TT_CAP < U <= WS_CAP products, one warp per row, by a sort instead of a hash table: the row's
// products are formed once into shared memory (A entries 32 at a time, each lane writing the products
// of its entry in B-row order, so product t follows the (k, q) order), their keys
// ((column - the row's smallest column) << 8 | t) are bitonic-sorted across the warp, 32E keys held
// E per lane, and every run of equal columns is summed by the lane holding its first key: from 0.0,
// in ascending t, i.e. ascending intermediate index k (Gustavson's order, bit for bit the sums of
// the hash kernels and of the oracle).  Rows whose columns span 2^24 or more are listed for the hash
// kernels.  The sorted runs come out in column order, so no sort of the output follows.
constexpr int WS_CAP = 256;  // a sort of 32E keys, E <= 8 per lane (longer rows: the hash kernels)
constexpr int WS_WARPS = 4;

template <int E>
__device__ __forceinline__ void ws_sort(uint32_t (&key)[8], int lane) {
  constexpr int N = 32 * E;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < E) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pe = e ^ j;
          if (pe > e) {
            const int g = lane * E + e;
            const bool up = (g & k) == 0;
            const uint32_t a = key[e], b = key[pe];
            if ((a > b) == up) { key[e] = b; key[pe] = a; }
          }
        }
      } else {
        const int lm = j / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int g = lane * E + e;
          const uint32_t other = __shfl_xor_sync(0xffffffffu, key[e], lm);
          const bool up = (g & k) == 0;
          const bool lower = (g & j) == 0;
          // the lower position keeps the smaller key in an ascending run, the larger otherwise
          key[e] = (lower == up) ? min(key[e], other) : max(key[e], other);
        }
      }
    }
  }
}

template <int E>
__device__ __forceinline__ int ws_row(int lane, int U, int32_t cbase, int32_t* sc, const double* sv, uint32_t* sk,
                                      int32_t* __restrict__ ocol, double* __restrict__ oval) {
  uint32_t key[8];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int t = lane * E + e;
    key[e] = t < U ? ((uint32_t)(sc[t] - cbase) << 8) | (uint32_t)t : 0xFFFFFFFFu;
  }
  ws_sort<E>(key, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) sk[lane * E + e] = key[e];
  __syncwarp();
  // run heads among this lane's keys; their positions, in order, go to sc (the products' columns
  // are no longer needed: a key holds its column)
  int nh = 0;
  unsigned heads = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int g = lane * E + e;
    if (g < U && (g == 0 || (key[e] >> 8) != (sk[g - 1] >> 8))) { heads |= 1u << e; ++nh; }
  }
  int x = nh;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  int pos = x - nh;
  const int total = __shfl_sync(0xffffffffu, x, 31);
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (heads & (1u << e)) sc[pos++] = lane * E + e;
  __syncwarp();
  // one run per lane: the FP64 additions of 32 runs go in one instruction stream (a lane holding
  // several heads would walk its runs one after another while the other lanes idle)
  for (int h0 = 0; h0 < total; h0 += 32) {
    const int hh = h0 + lane;
    if (hh < total) {
      int g = sc[hh];
      const int end = hh + 1 < total ? sc[hh + 1] : U;
      const uint32_t k0 = sk[g];
      double acc = 0.0;
      for (; g < end; ++g) acc = __dadd_rn(acc, sv[sk[g] & 0xFFu]);
      ocol[hh] = cbase + (int32_t)(k0 >> 8);
      oval[hh] = acc;
    }
  }
  return total;
}

__global__ void __launch_bounds__(32 * WS_WARPS) k_spgemm_wsort(
    int64_t r0, int64_t m, int64_t sbase, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
    const double* __restrict__ av, const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
    const double* __restrict__ bv, const int64_t* __restrict__ ub, const int64_t* __restrict__ soff,
    int32_t* __restrict__ scol, double* __restrict__ sval, int64_t* __restrict__ cnt, int32_t* __restrict__ list,
    int* __restrict__ nlist, int cap) {
  __shared__ int32_t s_col[WS_WARPS][WS_CAP];
  __shared__ double s_val[WS_WARPS][WS_CAP];
  __shared__ uint32_t s_key[WS_WARPS][WS_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = r0 + (int64_t)blockIdx.x * WS_WARPS + w;
  if (i >= m) return;
  const int U = (int)ub[i];
  if (U <= TT_CAP || U > cap) return;  // k_spgemm_tiny; the hash kernels
  int32_t* sc = s_col[w];
  double* sv = s_val[w];
  // products in (k, q) order: product t at sc[t], sv[t]
  int32_t cmin = INT_MAX, cmax = INT_MIN;
  int base = 0;
  const int64_t a0 = arp[i], a1 = arp[i + 1];
  for (int64_t p0 = a0; p0 < a1; p0 += 32) {
    const int64_t p = p0 + lane;
    int len = 0;
    int64_t b0 = 0;
    double a = 0.0;
    if (p < a1) {
      const int32_t k = aci[p];
      b0 = brp[k];
      len = (int)(brp[k + 1] - b0);
      a = av[p];
    }
    int x = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    int t = base + x - len;
    for (int q = 0; q < len; ++q, ++t) {
      const int32_t j = bci[b0 + q];
      sc[t] = j;
      sv[t] = __dmul_rn(a, bv[b0 + q]);
      cmin = min(cmin, j);
      cmax = max(cmax, j);
    }
    base += __shfl_sync(0xffffffffu, x, 31);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cmin = min(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
    cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  }
  if ((int64_t)cmax - (int64_t)cmin >= (int64_t(1) << 24)) {  // keys would not fit: the hash kernels
    if (lane == 0) list[atomicAdd(nlist, 1)] = (int32_t)i;
    return;
  }
  __syncwarp();
  const int64_t o = soff[i] - sbase;
  int total;
  if (U <= 64) total = ws_row<2>(lane, U, cmin, sc, sv, s_key[w], scol + o, sval + o);
  else if (U <= 128) total = ws_row<4>(lane, U, cmin, sc, sv, s_key[w], scol + o, sval + o);
  else total = ws_row<8>(lane, U, cmin, sc, sv, s_key[w], scol + o, sval + o);
  if (lane == 0) cnt[i] = total;
}

// The rows of a batch with WS_CAP < U <= FUSE_CAP, four warps per block with 256-slot tables: the
// table is sized by the row's distinct columns, not by its products (the coarse-operator rows keep a
// small fraction of their products), so small tables keep many warps resident; a row whose distinct
// columns pass FZ_LIMIT (a 70 % load) is stopped and listed, like the rows k_spgemm_wsort cannot key,
// for the 1024-slot list kernel, whose overflow goes on to the 4096-slot one.
constexpr int FZ_WARPS = 4;
constexpr int FZ_CAPA = 128;
constexpr int FZ_SLOTS = 256;
constexpr int FZ_LIMIT = FZ_SLOTS * 7 / 10;

__global__ void __launch_bounds__(32 * FZ_WARPS, 8) k_spgemm_fused_chunk(
    int64_t r0, int64_t m, int64_t sbase, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, const double* __restrict__ av,
    const int64_t* __restrict__ brp, const int32_t* __restrict__ bci, const double* __restrict__ bv,
    const int64_t* __restrict__ ub, const int64_t* __restrict__ soff, int32_t* __restrict__ scol,
    double* __restrict__ sval, int64_t* __restrict__ cnt, int32_t* __restrict__ list, int* __restrict__ nlist,
    int lo) {
  __shared__ int32_t hk[FZ_WARPS][FZ_SLOTS];
  __shared__ double hv[FZ_WARPS][FZ_SLOTS];
  __shared__ int32_t sst[FZ_WARPS][FZ_CAPA + 1];
  __shared__ int64_t sbg[FZ_WARPS][FZ_CAPA];
  __shared__ double sa[FZ_WARPS][FZ_CAPA];
  __shared__ double gv[FZ_WARPS][32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = r0 + (int64_t)blockIdx.x * FZ_WARPS + w;
  if (i >= m) return;
  int U = (int)ub[i];
  if (U <= lo || U > FUSE_CAP) return;  // k_spgemm_tiny or k_spgemm_wsort; the symbolic path
  ChunkSmem sm{hk[w], hv[w], sst[w], sbg[w], sa[w], gv[w]};
  const bool done = chunk_row<FZ_SLOTS, FZ_CAPA, false, FZ_LIMIT>(i, U, arp, aci, av, brp, bci, bv, soff[i] - sbase,
                                                                   scol, sval, cnt, sm);
  if (!done && lane == 0) list[atomicAdd(nlist, 1)] = (int32_t)i;
}

// The listed rows, W warps per block with SLOTS hash slots each (dynamic shared memory), a fixed grid
// walking the list.
template <int SLOTS, int CAPA>
constexpr size_t chunk_warp_bytes() {
  return ((size_t)SLOTS * 8 + (size_t)CAPA * 16 + 32 * 8 + (size_t)SLOTS * 4 + (size_t)(CAPA + 1) * 4 + 15) / 16 * 16;
}

template <int W, int SLOTS, int CAPA, int LIMIT>
__global__ void __launch_bounds__(32 * W, 2) k_spgemm_chunk_list(
    const int32_t* __restrict__ rows, const int* __restrict__ nrows, int64_t sbase, const int64_t* __restrict__ arp,
    const int32_t* __restrict__ aci, const double* __restrict__ av, const int64_t* __restrict__ brp,
    const int32_t* __restrict__ bci, const double* __restrict__ bv, const int64_t* __restrict__ ub,
    const int64_t* __restrict__ soff, int32_t* __restrict__ scol, double* __restrict__ sval,
    int64_t* __restrict__ cnt, int32_t* __restrict__ over, int* __restrict__ nover) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int w = threadIdx.x >> 5;
  unsigned char* base = dsm + (size_t)w * chunk_warp_bytes<SLOTS, CAPA>();
  ChunkSmem sm;
  sm.V = reinterpret_cast<double*>(base);
  sm.sbg = reinterpret_cast<int64_t*>(base + (size_t)SLOTS * 8);
  sm.sa = reinterpret_cast<double*>(base + (size_t)SLOTS * 8 + (size_t)CAPA * 8);
  sm.gv = reinterpret_cast<double*>(base + (size_t)SLOTS * 8 + (size_t)CAPA * 16);
  sm.K = reinterpret_cast<int32_t*>(base + (size_t)SLOTS * 8 + (size_t)CAPA * 16 + 32 * 8);
  sm.sst = reinterpret_cast<int32_t*>(base + (size_t)SLOTS * 12 + (size_t)CAPA * 16 + 32 * 8);
  const int64_t nr = *nrows;
  if ((int64_t)blockIdx.x * W + w >= nr) return;
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < SLOTS; t += 32) { sm.K[t] = -1; sm.V[t] = 0.0; }
  __syncwarp();
  for (int64_t r = (int64_t)blockIdx.x * W + w; r < nr; r += (int64_t)gridDim.x * W) {
    const int64_t i = rows[r];
    const bool done = chunk_row<SLOTS, CAPA, true, LIMIT>(i, (int)ub[i], arp, aci, av, brp, bci, bv, soff[i] - sbase,
                                                          scol, sval, cnt, sm);
    if (!done && lane == 0) over[atomicAdd(nover, 1)] = (int32_t)i;
  }
}

template <int W, int SLOTS, int CAPA, int LIMIT>
static void launch_chunk_list(Ctx& c, const int32_t* rows, const int* nrows, int64_t sbase, const DCSR<double>& A,
                              const DCSR<double>& B, const int64_t* ub, const int64_t* soff, int32_t* scol,
                              double* sval, int64_t* cnt, int64_t max_rows, int32_t* over, int* nover) {
  const size_t bytes = (size_t)W * chunk_warp_bytes<SLOTS, CAPA>();
  static int set_dev = -1;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (set_dev != dev) {
    CU(cudaFuncSetAttribute(k_spgemm_chunk_list<W, SLOTS, CAPA, LIMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)bytes));
    set_dev = dev;
  }
  // a fixed grid: the list's length is known on the device only
  const unsigned grid = grid_for(max_rows, W, (int64_t)c.num_sms * 8);
  k_spgemm_chunk_list<W, SLOTS, CAPA, LIMIT><<<grid, 32 * W, bytes, c.s>>>(rows, nrows, sbase, A.rp, A.ci, A.v, B.rp,
                                                                           B.ci, B.v, ub, soff, scol, sval, cnt, over,
                                                                           nover);
  CU_LAUNCH();
}

// copy the staged columns and values of the fused rows to their final place in C
__global__ void k_spgemm_fused_copy(int64_t m, const int64_t* __restrict__ ub, const int64_t* __restrict__ soff,
                                    const int32_t* __restrict__ scol, const double* __restrict__ sval,
                                    const int64_t* __restrict__ crp, int32_t* __restrict__ cci,
                                    double* __restrict__ cv) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  int sub = threadIdx.x & 7;
  if (i >= m || ub[i] > FUSE_CAP) return;
  int64_t o = soff[i], c0 = crp[i], L = crp[i + 1] - c0;
  for (int64_t t = sub; t < L; t += 8) {
    cci[c0 + t] = scol[o + t];
    cv[c0 + t] = sval[o + t];
  }
}
// Batches of the fused rows: batch b starts at the first row whose staging offset reaches
// b * budget (offsets grow by at most FUSE_CAP < budget per row, so every batch has a first row).
__global__ void k_batch_starts(int64_t m, const int64_t* soff, int64_t budget, int64_t* bstart, int64_t* bbase) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t b = soff[i] / budget;
  if (i == 0 || soff[i - 1] / budget != b) { bstart[b] = i; bbase[b] = soff[i]; }
}
__global__ void k_batch_counts(int64_t i0, int64_t i1, const int64_t* ub, const int64_t* cnt, int64_t* pc) {
  int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < i1) pc[i - i0] = ub[i] <= FUSE_CAP ? cnt[i] : 0;
}
// staged rows of one batch -> packed (exact sizes), and packed -> their rows of C
__global__ void k_batch_pack(int64_t i0, int64_t i1, const int64_t* ub, const int64_t* soff, int64_t sbase,
                             const int32_t* scol, const double* sval, const int64_t* poff, int32_t* pcol, double* pval) {
  int64_t i = i0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3);
  int sub = threadIdx.x & 7;
  if (i >= i1 || ub[i] > FUSE_CAP) return;
  int64_t o = soff[i] - sbase, d = poff[i - i0], L = poff[i - i0 + 1] - d;
  for (int64_t t = sub; t < L; t += 8) { pcol[d + t] = scol[o + t]; pval[d + t] = sval[o + t]; }
}
__global__ void k_batch_unpack(int64_t i0, int64_t i1, const int64_t* ub, const int64_t* poff, const int32_t* pcol,
                               const double* pval, const int64_t* crp, int32_t* cci, double* cv) {
  int64_t i = i0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3);
  int sub = threadIdx.x & 7;
  if (i >= i1 || ub[i] > FUSE_CAP) return;
  int64_t d = poff[i - i0], c0 = crp[i], L = crp[i + 1] - c0;
  for (int64_t t = sub; t < L; t += 8) { cci[c0 + t] = pcol[d + t]; cv[c0 + t] = pval[d + t]; }
}

__global__ void k_small_ub(int64_t m, const int64_t* ub, int64_t* us) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) us[i] = ub[i] <= FUSE_CAP ? ub[i] : 0;
}

void spgemm(Ctx& c, const DCSR<double>& A, const DCSR<double>& B, DCSR<double>& C, const char* name, bool sort_rows) {
  // rows of TT_CAP < U <= cap products take the sort kernel, longer ones the hash kernels
  const int sort_cap = sort_rows ? WS_CAP : TT_CAP;
  if (A.nc != B.nr) throw Error(MGR_ERR_INVALID_ARG, "spgemm: inner dimensions differ");
  int64_t m = A.nr;
  C.nr = m;
  C.nc = B.nc;
  C.rp.alloc(c, m + 1);
  if (m == 0) {
    fill_i64(c, C.rp.p, 0, 1);
    C.nnz = 0;
    C.ci.alloc(c, 0);
    C.v.alloc(c, 0);
    return;
  }
  ProfScope ps(c, "spgemm");
  ProfScope psn(c, name);
  DBuf<int64_t> ub(c, m), cnt(c, m + 1), us(c, m + 1);
  DBuf<int32_t> mid(c, m), big(c, m);
  DBuf<int> counters(c, 2);
  CU(cudaMemsetAsync(counters.p, 0, 2 * sizeof(int), c.s));
  {
    ProfScope ps1(c, "sym_ub");
    k_spgemm_ub<<<grid_for(m, 256), 256, 0, c.s>>>(m, A.rp, A.ci, B.rp, ub.p, counters.p, mid.p, counters.p + 1, big.p);
    CU_LAUNCH();
    k_small_ub<<<grid_for(m, 256), 256, 0, c.s>>>(m, ub.p, us.p);
    CU_LAUNCH();
  }
  DBuf<int64_t> soff(c, m + 1);
  scan_excl_i64(c, us.p, soff.p, m);
  // one wait for the staged total and the two row classes of the symbolic pass
  int64_t nstage = 0;
  int hc[2] = {0, 0};
  read_back(c, {{soff.p + m, &nstage, sizeof(int64_t)}, {counters.p, &hc[0], sizeof(int)},
                {counters.p + 1, &hc[1], sizeof(int)}});
  // the fused rows are staged (up to their product count each) in batches of at most
  // stage + FUSE_CAP entries; with several batches, each is packed to its exact size before
  // the next one is staged, so the transient memory follows the output, not the product count
  const int64_t stage = c.spgemm_stage > FUSE_CAP ? c.spgemm_stage : SPGEMM_STAGE;
  const int64_t nbatch = nstage / stage + 1;
  std::vector<int64_t> bst(nbatch + 1, m), bbase(nbatch + 1, nstage);
  if (nbatch > 1) {
    DBuf<int64_t> dbs(c, nbatch), dbb(c, nbatch);
    fill_i64(c, dbs.p, m, nbatch);  // a batch without a first row stays empty
    fill_i64(c, dbb.p, nstage, nbatch);
    k_batch_starts<<<grid_for(m, 256), 256, 0, c.s>>>(m, soff.p, stage, dbs.p, dbb.p);
    CU_LAUNCH();
    CU(cudaMemcpyAsync(bst.data(), dbs.p, sizeof(int64_t) * nbatch, cudaMemcpyDeviceToHost, c.s));
    CU(cudaMemcpyAsync(bbase.data(), dbb.p, sizeof(int64_t) * nbatch, cudaMemcpyDeviceToHost, c.s));
    host_wait(c);
    for (int64_t b = nbatch - 1; b >= 0; --b) {
      bst[b] = std::min(bst[b], bst[b + 1]);
      bbase[b] = std::min(bbase[b], bbase[b + 1]);
    }
  } else {
    bst[0] = 0;
    bbase[0] = 0;
  }
  int64_t cap = 0;
  for (int64_t b = 0; b < nbatch; ++b) cap = std::max(cap, bbase[b + 1] - bbase[b]);
  DBuf<int32_t> scol(c, cap + 1);
  DBuf<double> sval(c, cap + 1);
  std::vector<DBuf<int64_t>> poff(nbatch > 1 ? nbatch : 0);
  std::vector<DBuf<int32_t>> pcol(poff.size());
  std::vector<DBuf<double>> pval(poff.size());
  DBuf<int32_t> lists(c, 2 * m);
  DBuf<int> nlist(c, 2);
  for (int64_t b = 0; b < nbatch; ++b) {
    const int64_t i0 = bst[b], i1 = bst[b + 1], base = bbase[b];
    if (i1 <= i0) continue;
    {
      ProfScope ps2(c, "fused_small");
      CU(cudaMemsetAsync(nlist.p, 0, 2 * sizeof(int), c.s));
      k_spgemm_tiny<<<grid_for(i1 - i0, TT_THREADS), TT_THREADS, 0, c.s>>>(i0, i1, base, A.rp, A.ci, A.v, B.rp, B.ci,
                                                                           B.v, ub.p, soff.p, scol.p, sval.p, cnt.p);
      CU_LAUNCH();
      if (sort_cap > TT_CAP) {
        k_spgemm_wsort<<<grid_for(i1 - i0, WS_WARPS), 32 * WS_WARPS, 0, c.s>>>(
            i0, i1, base, A.rp, A.ci, A.v, B.rp, B.ci, B.v, ub.p, soff.p, scol.p, sval.p, cnt.p, lists.p, nlist.p, sort_cap);
        CU_LAUNCH();
      }
      k_spgemm_fused_chunk<<<grid_for(i1 - i0, FZ_WARPS), 32 * FZ_WARPS, 0, c.s>>>(
          i0, i1, base, A.rp, A.ci, A.v, B.rp, B.ci, B.v, ub.p, soff.p, scol.p, sval.p, cnt.p, lists.p, nlist.p, sort_cap);
      CU_LAUNCH();
      launch_chunk_list<4, 1024, 256, 1024 * 7 / 10>(c, lists.p, nlist.p, base, A, B, ub.p, soff.p, scol.p, sval.p,
                                                     cnt.p, i1 - i0, lists.p + m, nlist.p + 1);
      launch_chunk_list<1, 4096, 512, 4096>(c, lists.p + m, nlist.p + 1, base, A, B, ub.p, soff.p, scol.p, sval.p,
                                            cnt.p, i1 - i0, nullptr, nullptr);
    }
    if (nbatch > 1) {
      ProfScope ps3(c, "fused_copy");
      int64_t nr = i1 - i0;
      DBuf<int64_t> pc(c, nr + 1);
      k_batch_counts<<<grid_for(nr, 256), 256, 0, c.s>>>(i0, i1, ub.p, cnt.p, pc.p);
      CU_LAUNCH();
      poff[b].alloc(c, nr + 1);
      int64_t tot = counts_to_rowptr(c, pc.p, poff[b].p, nr);
      pcol[b].alloc(c, tot + 1);
      pval[b].alloc(c, tot + 1);
      k_batch_pack<<<grid_for(nr * 8, 256), 256, 0, c.s>>>(i0, i1, ub.p, soff.p, base, scol.p, sval.p, poff[b].p,
                                                           pcol[b].p, pval[b].p);
      CU_LAUNCH();
    }
  }
  if (nbatch > 1) {  // the staging is no longer needed
    scol.release();
    sval.release();
  }
  sym_pass(c, 0, A, B, mid.p, hc[0], big.p, hc[1], cnt.p, C);
  C.nnz = counts_to_rowptr(c, cnt.p, C.rp.p, m);
  C.ci.alloc(c, C.nnz);
  C.v.alloc(c, C.nnz);
  sym_pass(c, 1, A, B, mid.p, hc[0], big.p, hc[1], nullptr, C);
  {
    ProfScope ps3(c, "fused_copy");
    if (nbatch == 1) {
      k_spgemm_fused_copy<<<grid_for(m * 8, 256), 256, 0, c.s>>>(m, ub.p, soff.p, scol.p, sval.p, C.rp.p, C.ci.p,
                                                                   C.v.p);
      CU_LAUNCH();
    } else {
      for (int64_t b = 0; b < nbatch; ++b) {
        const int64_t i0 = bst[b], i1 = bst[b + 1];
        if (i1 <= i0) continue;
        k_batch_unpack<<<grid_for((i1 - i0) * 8, 256), 256, 0, c.s>>>(i0, i1, ub.p, poff[b].p, pcol[b].p, pval[b].p,
                                                                       C.rp.p, C.ci.p, C.v.p);
        CU_LAUNCH();
        pcol[b].release();
        pval[b].release();
      }
    }
  }
  if (c.prof && c.prof->wants(name)) {
    // algorithmic bytes of the product: A once, one B entry (column, value) per product, C written
    DBuf<int64_t> pp(c, m + 1);
    int64_t products = counts_to_rowptr(c, ub.p, pp.p, m);
    prof_add_bytes(c, name, 12.0 * (double)(A.nnz + products + C.nnz) + 16.0 * (double)(m + 1));
  }
  // the numeric pass of the rows over FUSE_CAP products (none in most products: no launch then)
  if (hc[0] + hc[1] > 0) {
    ProfScope ps4(c, "spgemm_numeric");
    k_spgemm_numeric_expand<<<grid_for(C.nr, NX_WARPS), 32 * NX_WARPS, 0, c.s>>>(C.nr, A.rp, A.ci, A.v, B.rp, B.ci,
                                                                                  B.v, C.rp, C.ci, C.v, ub.p);
    CU_LAUNCH();
    k_spgemm_numeric<<<grid_for(C.nr, NUM_WARPS), 32 * NUM_WARPS, 0, c.s>>>(C.nr, A.rp, A.ci, A.v, B.rp, B.ci, B.v,
                                                                             C.rp, C.ci, C.v, ub.p);
    CU_LAUNCH();
  }
}

// ---------------------------------------------------------------------------------------------
// Per-row sort of (column, value) pairs by column: a warp per row up to SORT_WCAP entries, a block
// per row up to SORT_BCAP, and an insertion sort in global memory beyond (rare, slow, correct).
constexpr int SORT_WCAP = 512;
constexpr int SORT_WARPS = 4;
constexpr int SORT_BCAP = 4096;

template <bool HASV>
__device__ __forceinline__ void cmpswap(int32_t* key, double* val, int t, int x, bool up) {
  int32_t a = key[t], b = key[x];
  if ((a > b) == up) {
    key[t] = b; key[x] = a;
    if (HASV) { double va = val[t]; val[t] = val[x]; val[x] = va; }
  }
}

template <bool HASV>
__global__ void __launch_bounds__(32 * SORT_WARPS) k_sort_rows_warp(int64_t nr, const int64_t* rp, int32_t* ci, double* v,
                                                                    int* n_big, int32_t* big) {
  __shared__ int32_t sk[SORT_WARPS][SORT_WCAP];
  __shared__ double sv[SORT_WARPS][HASV ? SORT_WCAP : 1];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * SORT_WARPS + w;
  if (i >= nr) return;
  int64_t b = rp[i];
  int L = (int)(rp[i + 1] - b);
  if (L <= 1) return;
  if (L > SORT_WCAP) {
    if (lane == 0) big[atomicAdd(n_big, 1)] = (int32_t)i;
    return;
  }
  int n2 = next_pow2(L);
  for (int t = lane; t < n2; t += 32) {
    sk[w][t] = (t < L) ? ci[b + t] : INT_MAX;
    if (HASV) sv[w][t] = (t < L) ? v[b + t] : 0.0;
  }
  __syncwarp();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < n2; t += 32) {
        int x = t ^ j;
        if (x > t) cmpswap<HASV>(sk[w], sv[w], t, x, (t & k) == 0);
      }
      __syncwarp();
    }
  for (int t = lane; t < L; t += 32) {
    ci[b + t] = sk[w][t];
    if (HASV) v[b + t] = sv[w][t];
  }
}

template <bool HASV>
__device__ void sort_row_block(int64_t i, const int64_t* rp, int32_t* ci, double* v, int32_t* sk, double* sv) {
  int64_t b = rp[i];
  int L = (int)(rp[i + 1] - b);
  if (L > SORT_BCAP) {
    // insertion sort in place (single thread): correct for any length
    if (threadIdx.x == 0)
      for (int a = 1; a < L; ++a) {
        int32_t key = ci[b + a];
        double val = HASV ? v[b + a] : 0.0;
        int t = a - 1;
        while (t >= 0 && ci[b + t] > key) {
          ci[b + t + 1] = ci[b + t];
          if (HASV) v[b + t + 1] = v[b + t];
          --t;
        }
        ci[b + t + 1] = key;
        if (HASV) v[b + t + 1] = val;
      }
    return;
  }
  int n2 = next_pow2(L);
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    sk[t] = (t < L) ? ci[b + t] : INT_MAX;
    if (HASV) sv[t] = (t < L) ? v[b + t] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        int x = t ^ j;
        if (x > t) cmpswap<HASV>(sk, sv, t, x, (t & k) == 0);
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    ci[b + t] = sk[t];
    if (HASV) v[b + t] = sv[t];
  }
}

// The rows listed by the warp kernel, *nrows of them (a count on the device, so the host does not
// wait for it): blocks stride over the list.
template <bool HASV>
__global__ void k_sort_rows_block(const int32_t* rows, const int* nrows, const int64_t* rp, int32_t* ci, double* v) {
  extern __shared__ unsigned char sm_raw[];
  int32_t* sk = reinterpret_cast<int32_t*>(sm_raw);
  double* sv = reinterpret_cast<double*>(sm_raw + sizeof(int32_t) * SORT_BCAP);
  const int nr = *nrows;
  for (int r = blockIdx.x; r < nr; r += gridDim.x) {
    sort_row_block<HASV>(rows[r], rp, ci, v, sk, sv);
    __syncthreads();  // the next row reuses the shared arrays
  }
}

void sort_rows(Ctx& c, int64_t nr, const int64_t* rp, int32_t* ci, double* v) {
  if (nr <= 0) return;
  DBuf<int> nbig(c, 1);
  DBuf<int32_t> big(c, nr);
  CU(cudaMemsetAsync(nbig.p, 0, sizeof(int), c.s));
  if (v)
    k_sort_rows_warp<true><<<grid_for(nr, SORT_WARPS), 32 * SORT_WARPS, 0, c.s>>>(nr, rp, ci, v, nbig.p, big.p);
  else
    k_sort_rows_warp<false><<<grid_for(nr, SORT_WARPS), 32 * SORT_WARPS, 0, c.s>>>(nr, rp, ci, v, nbig.p, big.p);
  CU_LAUNCH();
  // rows over the warp kernel's cap (rare): a block each, launched without reading their count
  const size_t sh = (sizeof(int32_t) + sizeof(double)) * SORT_BCAP;
  const unsigned g = (unsigned)(nr < c.num_sms ? nr : c.num_sms);
  if (v) {
    CU(cudaFuncSetAttribute(k_sort_rows_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_sort_rows_block<true><<<g, 512, sh, c.s>>>(big.p, nbig.p, rp, ci, v);
  } else {
    CU(cudaFuncSetAttribute(k_sort_rows_block<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_sort_rows_block<false><<<g, 512, sh, c.s>>>(big.p, nbig.p, rp, ci, v);
  }
  CU_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// Transpose: column counts (atomic), scan, scatter to atomic slots, then per-row sort by column.
// Every (row, column) pair is unique, so the sorted result is independent of the scatter order.
__global__ void k_col_count(int64_t nnz, const int32_t* ci, unsigned long long* cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[k]], 1ull);
}
__global__ void k_transpose_scatter(int64_t nr, const int64_t* rp, const int32_t* ci, const double* v,
                                    const int64_t* trp, unsigned long long* slot, int32_t* tci, double* tv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nr) return;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    int32_t j = ci[k];
    int64_t d = trp[j] + (int64_t)atomicAdd(&slot[j], 1ull);
    tci[d] = (int32_t)i;
    if (v) tv[d] = v[k];
  }
}

void transpose(Ctx& c, const DCSR<double>& A, DCSR<double>& T) {
  T.nr = A.nc;
  T.nc = A.nr;
  T.nnz = A.nnz;
  T.rp.alloc(c, T.nr + 1);
  T.ci.alloc(c, T.nnz);
  bool hv = A.v.p != nullptr;
  if (hv) T.v.alloc(c, T.nnz);
  DBuf<unsigned long long> cnt(c, T.nr + 1);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (T.nr + 1), c.s));
  if (A.nnz > 0) {
    k_col_count<<<grid_for(A.nnz, 256, 8192), 256, 0, c.s>>>(A.nnz, A.ci, cnt.p);
    CU_LAUNCH();
  }
  scan_excl_i64(c, reinterpret_cast<const int64_t*>(cnt.p), T.rp.p, T.nr);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (T.nr + 1), c.s));
  if (A.nr > 0) {
    k_transpose_scatter<<<grid_for(A.nr, 256), 256, 0, c.s>>>(A.nr, A.rp, A.ci, hv ? A.v.p : nullptr, T.rp.p, cnt.p,
                                                              T.ci.p, hv ? T.v.p : nullptr);
    CU_LAUNCH();
  }
  sort_rows(c, T.nr, T.rp.p, T.ci.p, hv ? T.v.p : nullptr);
}

// ---------------------------------------------------------------------------------------------
__global__ void k_f64_to_f32(int64_t n, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

void csr_to_f32(Ctx& c, const DCSR<double>& A, DCSR<float>& B) {
  B.nr = A.nr; B.nc = A.nc; B.nnz = A.nnz;
  B.rp.alloc(c, A.nr + 1);
  B.ci.alloc(c, A.nnz);
  B.v.alloc(c, A.nnz);
  CU(cudaMemcpyAsync(B.rp.p, A.rp.p, sizeof(int64_t) * (A.nr + 1), cudaMemcpyDeviceToDevice, c.s));
  if (A.nnz) {
    CU(cudaMemcpyAsync(B.ci.p, A.ci.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, c.s));
    k_f64_to_f32<<<grid_for(A.nnz, 256, 8192), 256, 0, c.s>>>(A.nnz, A.v.p, B.v.p);
    CU_LAUNCH();
  }
}

// B = the rows rows[0..nr) of A, in that order (pattern and values copied)
__global__ void k_gather_rows_count(int64_t nr, const int32_t* rows, const int64_t* rp, int64_t* cnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < nr) cnt[r] = rp[rows[r] + 1] - rp[rows[r]];
}
__global__ void k_gather_rows_fill(int64_t nr, const int32_t* rows, const int64_t* rp, const int32_t* ci,
                                   const double* v, const int64_t* orp, int32_t* oci, double* ov) {
  int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  int sub = threadIdx.x & 7;
  if (r >= nr) return;
  int64_t b = rp[rows[r]], e = rp[rows[r] + 1], o = orp[r];
  for (int64_t k = b + sub; k < e; k += 8) {
    oci[o + (k - b)] = ci[k];
    ov[o + (k - b)] = v[k];
  }
}
void csr_gather_rows(Ctx& c, const DCSR<double>& A, const int32_t* rows, int64_t nr, DCSR<double>& B, int64_t nnz) {
  DBuf<int64_t> cnt(c, nr + 1);
  B.nr = nr;
  B.nc = A.nc;
  B.rp.alloc(c, nr + 1);
  if (nr > 0) {
    k_gather_rows_count<<<grid_for(nr, 256), 256, 0, c.s>>>(nr, rows, A.rp, cnt.p);
    CU_LAUNCH();
  }
  if (nnz >= 0) {
    scan_excl_i64(c, cnt.p, B.rp.p, nr);
    B.nnz = nnz;
  } else {
    B.nnz = counts_to_rowptr(c, cnt.p, B.rp.p, nr);
  }
  B.ci.alloc(c, B.nnz);
  B.v.alloc(c, B.nnz);
  if (nr > 0) {
    k_gather_rows_fill<<<grid_for(nr * 8, 256), 256, 0, c.s>>>(nr, rows, A.rp, A.ci, A.v, B.rp, B.ci, B.v);
    CU_LAUNCH();
  }
}

void copy_csr(Ctx& c, const DCSR<double>& A, DCSR<double>& B) {
  B.nr = A.nr; B.nc = A.nc; B.nnz = A.nnz;
  B.rp.alloc(c, A.nr + 1);
  B.ci.alloc(c, A.nnz);
  CU(cudaMemcpyAsync(B.rp.p, A.rp.p, sizeof(int64_t) * (A.nr + 1), cudaMemcpyDeviceToDevice, c.s));
  if (A.nnz) CU(cudaMemcpyAsync(B.ci.p, A.ci.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, c.s));
  if (A.v.p) {
    B.v.alloc(c, A.nnz);
    if (A.nnz) CU(cudaMemcpyAsync(B.v.p, A.v.p, sizeof(double) * A.nnz, cudaMemcpyDeviceToDevice, c.s));
  }
}

}  // namespace mgr
