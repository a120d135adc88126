// sort.cu -- particles into cell order (the sort of Alg. 1 / Alg. 2's
// sort_and_calc_moments step): a stable least-significant-digit radix sort of
// the particles' cell indices, the CSR cell offsets, and the gather of the
// velocities into the sorted order.
//
// Keys are cell indices; an index outside [0, n_cells) becomes n_cells, so
// such particles (left the domain, say) end up behind the last cell and
// belong to no cell.  The key has B = bit_length(n_cells) bits, sorted in
// P = ceil(B / 9) passes of ceil(B / P) bits each (two passes up to 2^18
// cells).  One pass:
//   * radix_hist_kernel: each tile of 4096 keys counts its digits into
//     counts[digit][tile] (digit-major), one shared-memory atomic per
//     distinct digit of a warp (match_any);
//   * an exclusive scan of counts (three kernels) gives every (digit, tile)
//     its first output position;
//   * radix_scatter_kernel: each warp ranks a strip of 256 consecutive keys
//     of the tile stably, 32 at a time (match_any, a per-warp running count
//     per digit); one block-wide step turns the per-warp counts into offsets;
//     the tile is placed sorted by digit in shared memory and each digit's
//     run written to its position, so stores are contiguous runs.
// Ranks only count keys that come earlier in the input, so equal keys keep
// their input order: the result is the stable permutation, the same on
// every run.
#include <cstdint>

#include "fp_device.cuh"

namespace fpc {

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                          // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys per tile
constexpr int kWarpStrip = kSortTile / kSortWarps;     // 256 consecutive keys per warp
constexpr int kMaxBits = 9;
constexpr int kMaxRadix = 1 << kMaxBits;

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 entries per scan block

__device__ __forceinline__ uint32_t cell_key(int32_t c, int64_t n_cells) {
  return (c >= 0 && (int64_t)c < n_cells) ? (uint32_t)c : (uint32_t)n_cells;
}

template <bool kFirst>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const int32_t *__restrict__ cell_of,
                                                                  const uint32_t *__restrict__ keys, int64_t n,
                                                                  int64_t n_cells, int shift, int bits,
                                                                  int64_t n_tiles, uint32_t *__restrict__ counts) {
  __shared__ uint32_t h[kMaxRadix];
  const int radix = 1 << bits;
  for (int d = threadIdx.x; d < radix; d += kSortThreads) h[d] = 0u;
  __syncthreads();
  // each warp counts a strip of consecutive keys 32 at a time (coalesced
  // loads); a lane whose digit differs from its left neighbour's starts a
  // run, and each run adds its length with one shared-memory atomic
  // (cell-ordered input has long runs)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t s0 = (int64_t)blockIdx.x * kSortTile + (int64_t)w * kWarpStrip;
  uint32_t k[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = s0 + r * 32 + lane;
    k[r] = i < n ? (kFirst ? cell_key(cell_of[i], n_cells) : keys[i]) : 0xffffffffu;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = k[r] != 0xffffffffu;
    const uint32_t d = valid ? (k[r] >> shift) & (uint32_t)(radix - 1) : (uint32_t)kMaxRadix;
    const uint32_t dl = __shfl_up_sync(0xffffffffu, d, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || d != dl);
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    if (valid && ((starts >> lane) & 1u)) {
      const unsigned after = starts & ~((2u << lane) - 1u);  // run starts above this lane (lane 31: none)
      const int end = lane == 31 ? 32 : (after ? __ffs(after) - 1 : 32);
      const int last = 32 - __clz(vmask);                   // valid lanes are 0 .. last - 1
      atomicAdd(&h[d], (uint32_t)((end < last ? end : last) - lane));
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += kSortThreads) counts[(int64_t)d * n_tiles + blockIdx.x] = h[d];
}

// Exclusive scan of the block's kScanTile entries held kScanItems per thread
// (blocked); returns the block total.  `carry` is added to every output.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t (&x)[kScanItems], uint32_t carry,
                                                         uint32_t *warp_tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) s += x[j];
  uint32_t inc = s;  // inclusive scan of the thread sums across the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) warp_tot[kScanThreads / 32] = ti;       // block total
  }
  __syncthreads();
  uint32_t run = carry + warp_tot[w] + inc - s;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint32_t v = x[j];
    x[j] = run;
    run += v;
  }
  const uint32_t total = warp_tot[kScanThreads / 32];
  __syncthreads();  // warp_tot is reused by the caller's next scan
  return total;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *__restrict__ x, int64_t len,
                                                                   uint32_t *__restrict__ block_sums) {
  __shared__ uint32_t red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
    if (i < len) s += x[i];
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0u;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the block sums in place, kScanTile at a time.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(uint32_t *__restrict__ sums, int64_t nb) {
  __shared__ uint32_t warp_tot[kScanThreads / 32 + 1];
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanTile) {
    uint32_t x[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
      x[j] = i < nb ? sums[i] : 0u;
    }
    const uint32_t tot = block_exclusive_scan(x, carry, warp_tot);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
      if (i < nb) sums[i] = x[j];
    }
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(uint32_t *__restrict__ x, int64_t len,
                                                                 const uint32_t *__restrict__ block_offsets) {
  __shared__ uint32_t warp_tot[kScanThreads / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
    v[j] = i < len ? x[i] : 0u;
  }
  block_exclusive_scan(v, block_offsets[blockIdx.x], warp_tot);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + (int64_t)threadIdx.x * kScanItems + j;
    if (i < len) x[i] = v[j];
  }
}

template <bool kFirst>
__global__ void __launch_bounds__(kSortThreads, 2) radix_scatter_kernel(
    const int32_t *__restrict__ cell_of, const uint32_t *__restrict__ keys_in, const int32_t *__restrict__ idx_in,
    int64_t n, int64_t n_cells, int shift, int bits, int64_t n_tiles, const uint32_t *__restrict__ pos,
    uint32_t *__restrict__ keys_out, int32_t *__restrict__ idx_out) {
  // the per-warp digit counts are dead once every key knows its place, so
  // the tile staged sorted by digit reuses their memory
  constexpr int kCountBytes = kSortWarps * kMaxRadix * 2, kStageBytes = kSortTile * 8;
  __shared__ __align__(16) unsigned char raw[kCountBytes > kStageBytes ? kCountBytes : kStageBytes];
  uint16_t(*wc)[kMaxRadix] = reinterpret_cast<uint16_t(*)[kMaxRadix]>(raw);  // per warp: keys of each digit
  uint32_t *sk = reinterpret_cast<uint32_t *>(raw);
  int32_t *si = reinterpret_cast<int32_t *>(raw + kSortTile * 4);
  __shared__ uint32_t lstart[kMaxRadix];  // tile-local start of each digit
  __shared__ int32_t gbase[kMaxRadix];    // output position of the tile's digit d, minus lstart[d]
  const int radix = 1 << bits;
  const uint32_t mask = (uint32_t)(radix - 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kMaxRadix; d += kSortThreads) {
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) wc[q][d] = 0;
  }
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t s0 = t0 + (int64_t)w * kWarpStrip;  // this warp's strip
  uint32_t key[kSortItems];
  int32_t idx[kSortItems];
  uint16_t rank[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {  // all loads first
    const int64_t i = s0 + r * 32 + lane;
    key[r] = 0u;
    idx[r] = 0;
    if (i < n) {
      key[r] = kFirst ? cell_key(cell_of[i], n_cells) : keys_in[i];
      idx[r] = kFirst ? (int32_t)i : idx_in[i];
    }
  }
  // warp-local stable ranks: key s0 + 32 r + lane comes after every key of
  // rounds < r and after the lanes below it with the same digit
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = s0 + r * 32 + lane;
    const bool valid = i < n;
    const uint32_t d = valid ? (key[r] >> shift) & mask : (uint32_t)kMaxRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t base = valid ? wc[w][d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wc[w][d] = (uint16_t)(base + __popc(peers));
    __syncwarp();
    rank[r] = (uint16_t)(base + __popc(peers & ((1u << lane) - 1u)));
  }
  __syncthreads();
  // per digit: the warps' exclusive offsets (in place) and the tile total
  for (int d = threadIdx.x; d < radix; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) {
      const uint32_t c = wc[q][d];
      wc[q][d] = (uint16_t)run;
      run += c;
    }
    lstart[d] = run;
  }
  __syncthreads();
  if (w == 0) {  // exclusive scan of the digit totals
    uint32_t carry = 0;
    for (int b = 0; b < radix; b += 32) {
      const uint32_t x = b + lane < radix ? lstart[b + lane] : 0u;
      uint32_t inc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (b + lane < radix) lstart[b + lane] = carry + inc - x;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += kSortThreads)
    gbase[d] = (int32_t)((int64_t)pos[(int64_t)d * n_tiles + blockIdx.x] - (int64_t)lstart[d]);
  uint32_t lp[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t d = (key[r] >> shift) & mask;
    lp[r] = lstart[d] + wc[w][d] + rank[r];
  }
  __syncthreads();  // the counts are read; their memory becomes the staging tile
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = s0 + r * 32 + lane;
    if (i < n) {
      sk[lp[r]] = key[r];
      si[lp[r]] = idx[r];
    }
  }
  __syncthreads();
  const int cnt = (int)(n - t0 < kSortTile ? n - t0 : kSortTile);
  for (int k = threadIdx.x; k < cnt; k += kSortThreads) {
    const uint32_t d = (sk[k] >> shift) & mask;
    const int64_t g = (int64_t)gbase[d] + k;
    if (g >= 0 && g < n) {  // always true for a consistent count / scan; keeps every store in bounds
      keys_out[g] = sk[k];
      idx_out[g] = si[k];
    }
  }
}

// offsets[c] = first sorted position whose key is >= c, for c in [0, n_cells];
// each thread takes 8 consecutive positions (positions 0..n, n meaning "past
// the end" with key n_cells)
constexpr int kOffItems = 8;
__global__ void __launch_bounds__(256) cell_offsets_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                           int64_t n_cells, int64_t *__restrict__ offsets) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kOffItems;
  if (i0 > n) return;
  int64_t prev = i0 == 0 ? -1 : min((int64_t)keys[i0 - 1], n_cells);
#pragma unroll
  for (int j = 0; j < kOffItems; ++j) {
    const int64_t i = i0 + j;
    if (i > n) break;
    const int64_t cur = i == n ? n_cells : min((int64_t)keys[i], n_cells);
    for (int64_t c = prev + 1; c <= cur; ++c) offsets[c] = i;
    prev = cur;
  }
}

template <typename VT>
__global__ void __launch_bounds__(256) gather_sorted_kernel(const VT *__restrict__ v, int64_t n,
                                                            const int32_t *__restrict__ perm,
                                                            VT *__restrict__ v_sorted) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  if (p < 0 || p >= n) p = i;  // never taken for a permutation; keeps every load in bounds
  v_sorted[i] = v[p];
  v_sorted[n + i] = v[n + p];
  v_sorted[2 * n + i] = v[2 * n + p];
}

// v_out[d][i] = v[d][i] for i >= *first (the particles behind the last cell)
template <typename VT>
__global__ void __launch_bounds__(256) copy_tail_kernel(const VT *__restrict__ v, VT *__restrict__ v_out, int64_t n,
                                                        const int64_t *__restrict__ first) {
  const int64_t a = *first;
  for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    v_out[i] = v[i];
    v_out[n + i] = v[n + i];
    v_out[2 * n + i] = v[2 * n + i];
  }
}

void launch_copy_tail(const void *v, void *v_out, int v_dtype, int64_t n, const int64_t *first, cudaStream_t st) {
  if (n <= 0) return;
  if (v_dtype == FP_V_F32)
    copy_tail_kernel<float><<<304, 256, 0, st>>>((const float *)v, (float *)v_out, n, first);
  else
    copy_tail_kernel<double><<<304, 256, 0, st>>>((const double *)v, (double *)v_out, n, first);
}

static inline size_t sort_align(size_t x) { return (x + 255) & ~(size_t)255; }

struct SortPlan {
  int64_t n_tiles, counts_len, scan_blocks;
  int passes, bits[4];
  size_t off_keys0, off_keys1, off_idx0, off_idx1, off_counts, off_sums, total;
};

static SortPlan sort_plan(int64_t n, int64_t n_cells) {
  SortPlan P{};
  int B = 0;
  while (B < 32 && ((uint64_t)n_cells >> B) != 0) ++B;  // keys are 0..n_cells
  if (B == 0) B = 1;
  P.passes = (B + kMaxBits - 1) / kMaxBits;
  const int per = (B + P.passes - 1) / P.passes;
  int left = B;
  for (int q = 0; q < P.passes; ++q) {
    P.bits[q] = left < per ? left : per;
    left -= P.bits[q];
  }
  P.n_tiles = (n + kSortTile - 1) / kSortTile;
  if (P.n_tiles < 1) P.n_tiles = 1;
  P.counts_len = (int64_t)kMaxRadix * P.n_tiles;
  P.scan_blocks = (P.counts_len + kScanTile - 1) / kScanTile;
  size_t o = 0;
  P.off_keys0 = o;
  o += sort_align((size_t)n * 4);
  P.off_keys1 = o;
  o += sort_align((size_t)n * 4);
  P.off_idx0 = o;
  o += sort_align((size_t)n * 4);
  P.off_idx1 = o;
  o += sort_align((size_t)n * 4);
  P.off_counts = o;
  o += sort_align((size_t)P.counts_len * 4);
  P.off_sums = o;
  o += sort_align((size_t)P.scan_blocks * 4);
  P.total = o;
  return P;
}

size_t sort_workspace_bytes(int64_t n, int64_t n_cells) { return sort_plan(n, n_cells).total; }

// Sorted keys end in the returned buffer (nullptr on a bad workspace);
// perm (sorted position -> input index) and offsets are written.
void launch_sort_by_cell(const int32_t *cell_of, int64_t n, int64_t n_cells, int32_t *perm, int64_t *offsets,
                         void *ws, cudaStream_t st, const uint32_t **sorted_keys) {
  const SortPlan P = sort_plan(n, n_cells);
  char *w = (char *)ws;
  uint32_t *keys[2] = {(uint32_t *)(w + P.off_keys0), (uint32_t *)(w + P.off_keys1)};
  int32_t *idx[2] = {(int32_t *)(w + P.off_idx0), (int32_t *)(w + P.off_idx1)};
  uint32_t *counts = (uint32_t *)(w + P.off_counts);
  uint32_t *sums = (uint32_t *)(w + P.off_sums);
  int shift = 0, cur = 0;
  for (int q = 0; q < P.passes; ++q) {
    const int bits = P.bits[q];
    const int64_t len = (int64_t)(1 << bits) * P.n_tiles;
    const int64_t sblocks = (len + kScanTile - 1) / kScanTile;
    if (n > 0) {
      if (q == 0)
        radix_hist_kernel<true><<<(unsigned)P.n_tiles, kSortThreads, 0, st>>>(cell_of, nullptr, n, n_cells, shift,
                                                                               bits, P.n_tiles, counts);
      else
        radix_hist_kernel<false><<<(unsigned)P.n_tiles, kSortThreads, 0, st>>>(nullptr, keys[cur], n, n_cells,
                                                                                shift, bits, P.n_tiles, counts);
      scan_reduce_kernel<<<(unsigned)sblocks, kScanThreads, 0, st>>>(counts, len, sums);
      scan_top_kernel<<<1, kScanThreads, 0, st>>>(sums, sblocks);
      scan_down_kernel<<<(unsigned)sblocks, kScanThreads, 0, st>>>(counts, len, sums);
      // the last pass writes the permutation straight into perm
      int32_t *idx_dst = q == P.passes - 1 ? perm : idx[cur ^ 1];
      if (q == 0)
        radix_scatter_kernel<true><<<(unsigned)P.n_tiles, kSortThreads, 0, st>>>(
            cell_of, nullptr, nullptr, n, n_cells, shift, bits, P.n_tiles, counts, keys[cur ^ 1], idx_dst);
      else
        radix_scatter_kernel<false><<<(unsigned)P.n_tiles, kSortThreads, 0, st>>>(
            nullptr, keys[cur], idx[cur], n, n_cells, shift, bits, P.n_tiles, counts, keys[cur ^ 1], idx_dst);
    }
    cur ^= 1;
    shift += bits;
  }
  const int64_t blocks = (n + 1 + 256 * kOffItems - 1) / (256 * kOffItems);
  cell_offsets_kernel<<<(unsigned)blocks, 256, 0, st>>>(keys[cur], n, n_cells, offsets);
  if (sorted_keys) *sorted_keys = keys[cur];
}

void launch_gather_sorted(const void *v, int v_dtype, int64_t n, const int32_t *perm, void *v_sorted,
                          cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = (n + 255) / 256;
  if (v_dtype == FP_V_F32)
    gather_sorted_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float *)v, n, perm, (float *)v_sorted);
  else
    gather_sorted_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double *)v, n, perm, (double *)v_sorted);
}

}  // namespace fpc
