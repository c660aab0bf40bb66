// sell.cu -- construction of the sliced (SELL-32) layout of a 3x3 BSR matrix.
#include "bsr_sell.cuh"

namespace mgr {

__global__ void k_sell_width(int64_t nb, const int64_t* rp, int64_t nslices, int64_t* width) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t w = 0, e = (s + 1) * SELL_C < nb ? (s + 1) * SELL_C : nb;
  for (int64_t I = s * SELL_C; I < e; ++I) w = max(w, rp[I + 1] - rp[I]);
  width[s] = w;
}

__global__ void k_sell_fill_pattern(int64_t nb, int64_t nrows_padded, const int64_t* rp, const int32_t* ci,
                                    const int64_t* soff, int32_t* col, int64_t* src) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nrows_padded) return;
  int64_t s = I / SELL_C;
  int t = (int)(I - s * SELL_C);
  int64_t b0 = soff[s], b1 = soff[s + 1];
  int64_t len = I < nb ? rp[I + 1] - rp[I] : 0, k0 = I < nb ? rp[I] : 0;
  for (int64_t j = 0; j < b1 - b0; ++j) {
    int64_t slot = b0 + j;
    if (j < len) {
      col[slot * SELL_C + t] = ci[k0 + j];
      src[slot * SELL_C + t] = k0 + j;
    } else {
      col[slot * SELL_C + t] = (int32_t)(I < nb ? I : 0);
      src[slot * SELL_C + t] = -1;
    }
  }
}

void sell_build_pattern(Ctx& c, int64_t nb, int64_t nnzb, const int64_t* rowptr, const int32_t* colind,
                        SellPattern& S) {
  S.nb = nb;
  S.nnzb_real = nnzb;
  S.nslices = (nb + SELL_C - 1) / SELL_C;
  DBuf<int64_t> width(c, S.nslices + 1);
  k_sell_width<<<grid_for(S.nslices, 256), 256, 0, c.s>>>(nb, rowptr, S.nslices, width.p);
  CU_LAUNCH();
  S.soff.alloc(c, S.nslices + 1);
  S.slots = counts_to_rowptr(c, width.p, S.soff.p, S.nslices);
  S.col.alloc(c, S.slots * SELL_C);
  S.src.alloc(c, S.slots * SELL_C);
  int64_t np = S.nslices * SELL_C;
  k_sell_fill_pattern<<<grid_for(np, 256), 256, 0, c.s>>>(nb, np, rowptr, colind, S.soff.p, S.col.p, S.src.p);
  CU_LAUNCH();
}

// one thread per (slot, row-in-slice) pair; padding slots get zeros
template <class TS, class TD>
__global__ void k_sell_fill_values(int64_t n, const int64_t* __restrict__ src, const TS* __restrict__ v,
                                   TD* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  int64_t slot = idx / SELL_C;
  int t = (int)(idx - slot * SELL_C);
  int64_t k = src[idx];
  TD* o = out + slot * 9 * SELL_C + t;
#pragma unroll
  for (int e = 0; e < 9; ++e) o[e * SELL_C] = k >= 0 ? (TD)v[9 * k + e] : TD(0);
}

template <class TS, class TD>
void sell_fill_values(Ctx& c, const SellPattern& S, const TS* values, TD* out) {
  int64_t n = S.slots * SELL_C;
  if (n <= 0) return;
  k_sell_fill_values<TS, TD><<<grid_for(n, 256), 256, 0, c.s>>>(n, S.src.p, values, out);
  CU_LAUNCH();
}

template void sell_fill_values<double, double>(Ctx&, const SellPattern&, const double*, double*);
template void sell_fill_values<double, float>(Ctx&, const SellPattern&, const double*, float*);

__global__ void k_sell_compose(int64_t n, int64_t* src, const int64_t* perm) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n && src[idx] >= 0) src[idx] = perm[src[idx]];
}
void sell_compose_src(Ctx& c, SellPattern& S, const int64_t* perm) {
  int64_t n = S.slots * SELL_C;
  if (n <= 0) return;
  k_sell_compose<<<grid_for(n, 256), 256, 0, c.s>>>(n, S.src.p, perm);
  CU_LAUNCH();
}

template <class TS, class TD>
__global__ void k_sell_fill_values_t(int64_t n, const int64_t* __restrict__ src, const TS* __restrict__ v,
                                     TD* __restrict__ out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  int64_t slot = idx / SELL_C;
  int t = (int)(idx - slot * SELL_C);
  int64_t k = src[idx];
  TD* o = out + slot * 9 * SELL_C + t;
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) o[(3 * p + q) * SELL_C] = k >= 0 ? (TD)v[9 * k + 3 * q + p] : TD(0);
}

template <class TS, class TD>
void sell_fill_values_t(Ctx& c, const SellPattern& S, const TS* values, TD* out) {
  int64_t n = S.slots * SELL_C;
  if (n <= 0) return;
  k_sell_fill_values_t<TS, TD><<<grid_for(n, 256), 256, 0, c.s>>>(n, S.src.p, values, out);
  CU_LAUNCH();
}

template void sell_fill_values_t<double, double>(Ctx&, const SellPattern&, const double*, double*);
template void sell_fill_values_t<double, float>(Ctx&, const SellPattern&, const double*, float*);

}  // namespace mgr
