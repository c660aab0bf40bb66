// bsr_sell.cuh -- sliced layout of a 3x3 BSR matrix for coalesced sparse products.
//
// Block rows are grouped in slices of 32.  Slice s has width W_s = the longest block row in it and
// starts at slot B_s = W_0 + ... + W_{s-1}.  For slot j < W_s of row t of slice s:
//   col[(B_s + j) * 32 + t]               block column (the row itself for padding slots)
//   val[((B_s + j) * 9 + e) * 32 + t]     entry e = 3p + q of that block (0 for padding)
// so for every (slot, entry) the 32 rows of a slice are contiguous: one warp reads one 32-value line
// per load instruction, fully coalesced.  Padding is only the difference between the longest and
// the other rows of a slice (boundary rows of the grid).
#pragma once
#include "common.cuh"

namespace mgr {

constexpr int SELL_C = 32;

struct SellPattern {
  int64_t nb = 0, nslices = 0, slots = 0;
  int64_t nnzb_real = 0;  // stored blocks of the source matrix (slots * 32 minus padding)
  DBuf<int64_t> soff;  // nslices + 1 slot offsets
  DBuf<int32_t> col;   // slots * 32
  DBuf<int64_t> src;   // slots * 32: source block index in the BSR arrays, -1 for padding
};

// Builds the pattern of the sliced layout from a BSR pattern (rowptr, colind on the device).
void sell_build_pattern(Ctx& c, int64_t nb, int64_t nnzb, const int64_t* rowptr, const int32_t* colind,
                        SellPattern& S);
// Scatters BSR values (9 per block, row-major) into the sliced value layout (slots * 32 * 9).
template <class TS, class TD>
void sell_fill_values(Ctx& c, const SellPattern& S, const TS* values, TD* out);
// For the layout of A^T: src[] (positions in A^T's block order) replaced by perm[src] (A's blocks),
// and values filled with each source block transposed.
void sell_compose_src(Ctx& c, SellPattern& S, const int64_t* perm);
template <class TS, class TD>
void sell_fill_values_t(Ctx& c, const SellPattern& S, const TS* values, TD* out);

// Product over the sliced layout: one thread per block row; epi(I, s0, s1, s2) gets the row sums.
template <class T, class TX, class Epi>
__global__ void __launch_bounds__(256) k_bsr_sell(int64_t nb, const int64_t* __restrict__ soff,
                                                  const int32_t* __restrict__ col, const T* __restrict__ val,
                                                  const TX* __restrict__ x, Epi epi) {
  pdl_wait();
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  int64_t s = I / SELL_C;
  int t = (int)(I - s * SELL_C);
  int64_t b0 = soff[s], b1 = soff[s + 1];
  T s0 = 0, s1 = 0, s2 = 0;
  for (int64_t j = b0; j < b1; ++j) {
    int64_t J = col[j * SELL_C + t];
    const T* v = val + j * 9 * SELL_C + t;
    T x0 = (T)__ldg(x + 3 * J), x1 = (T)__ldg(x + 3 * J + 1), x2 = (T)__ldg(x + 3 * J + 2);
    // one FMA per product (FP64 instructions bound the FP64 variant on this GPU)
    s0 = fma(v[0 * SELL_C], x0, s0); s0 = fma(v[1 * SELL_C], x1, s0); s0 = fma(v[2 * SELL_C], x2, s0);
    s1 = fma(v[3 * SELL_C], x0, s1); s1 = fma(v[4 * SELL_C], x1, s1); s1 = fma(v[5 * SELL_C], x2, s1);
    s2 = fma(v[6 * SELL_C], x0, s2); s2 = fma(v[7 * SELL_C], x1, s2); s2 = fma(v[8 * SELL_C], x2, s2);
  }
  epi(I, s0, s1, s2);
}

template <class T, class TX, class Epi>
inline void launch_bsr_sell(Ctx& c, const SellPattern& S, const T* val, const TX* x, const Epi& epi) {
  launch_pdl(c, k_bsr_sell<T, TX, Epi>, grid_for(S.nb, 256), 256, 0, S.nb, S.soff.p, S.col.p, val, x, epi);
  CU_LAUNCH();
}

}  // namespace mgr
