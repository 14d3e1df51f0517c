// hm_sort.cu -- stable least-significant-digit radix sort of fixed-width int32 rows.
//
// Used twice on the path: to put the target's arcs in (src, dst) and (dst, src)
// order when a graph is loaded, and to put the output mappings in
// lexicographic order (original pattern-vertex columns) before they are
// returned.  The key is the concatenation of the chosen columns, each
// holding `bits` significant bits, most significant column first; it is
// consumed kDigitBits (10) bits per pass, so a 4-column key of 20-bit vertex
// ids takes 8 passes.
//
// One pass on a fixed grid of G blocks, block b owning the contiguous row
// range [b*R, (b+1)*R):
//   histogram  per-block digit counts               -> hist[digit * G + b]
//   scan       exclusive scan of hist               -> global start of each
//              (digit, block) bucket
//   scatter    the block walks its range in tiles of 1024 rows; inside a
//              tile each warp ranks its 4 rounds of 32 rows with
//              __match_any_sync, warps are ordered by an exclusive prefix over
//              their per-digit counts, so equal digits keep input order
//              (stability), the tile is reordered by digit in shared memory
//              and each digit's run is written by consecutive threads.
// Rows of four words (16-byte aligned, at least kFusedMinRows of them) run
// every pass in one cooperative launch (k_sort4_fused: the phases separated
// by grid-wide barriers); other widths and smaller sorts run each pass as
// five kernels (k_hist, three scan kernels, scatter).
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int kDigitBits = 10;
constexpr int kRadix = 1 << kDigitBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 4;
constexpr int kTile = kSortThreads * kItems;
constexpr int kMaxKeyCols = HM_MAX_K + 1;

struct KeySpec {
  int ncols;                 // key columns
  int cols[kMaxKeyCols];     // row word of each key column, most significant first
  int bits[kMaxKeyCols];     // significant bits of each key column (1..32)
  uint32_t xr[kMaxKeyCols];  // xor applied to a column before its bits are taken
  int shift;                 // bit position of this pass's digit within the whole key
  // the pass's digit as pieces of the columns it overlaps (set by set_pass):
  // digit |= ((word[tcol[t]] ^ txr[t]) >> tshr[t] & tmask[t]) << tshl[t]
  int nterm;
  int tcol[kMaxKeyCols], tshr[kMaxKeyCols], tshl[kMaxKeyCols];
  uint32_t tmask[kMaxKeyCols], txr[kMaxKeyCols];
};

// The pieces of the kDigitBits-bit digit starting at bit `shift` of the
// concatenated key (least significant column last in cols[]).
void set_pass(KeySpec &ks, int shift) {
  ks.shift = shift;
  ks.nterm = 0;
  int got = 0, col_lo = 0;
  for (int i = ks.ncols - 1; i >= 0 && got < kDigitBits; --i) {
    const int b = ks.bits[i];
    const int want_lo = shift + got;
    if (want_lo < col_lo + b) {
      const int r = want_lo - col_lo;
      const int take = std::min(b - r, kDigitBits - got);
      const int t = ks.nterm++;
      ks.tcol[t] = ks.cols[i];
      ks.tshr[t] = r;
      ks.tmask[t] = take >= 32 ? 0xffffffffu : ((1u << take) - 1u);
      ks.tshl[t] = got;
      ks.txr[t] = ks.xr[i];
      got += take;
    }
    col_lo += b;
  }
}

__device__ __forceinline__ uint32_t digit_of(const int32_t *__restrict__ row, const KeySpec &ks) {
  uint32_t v = 0;
  for (int t = 0; t < ks.nterm; ++t)
    v |= ((((uint32_t)__ldg(row + ks.tcol[t]) ^ ks.txr[t]) >> ks.tshr[t]) & ks.tmask[t]) << ks.tshl[t];
  return v;
}

// The same digit of a four-word row already in registers.
__device__ __forceinline__ uint32_t digit_of4(int4 r, const KeySpec &ks) {
  uint32_t v = 0;
  for (int t = 0; t < ks.nterm; ++t) {
    const int c = ks.tcol[t];
    const uint32_t col = (uint32_t)(c == 0 ? r.x : c == 1 ? r.y : c == 2 ? r.z : r.w) ^ ks.txr[t];
    v |= ((col >> ks.tshr[t]) & ks.tmask[t]) << ks.tshl[t];
  }
  return v;
}

// A pass's digit over four-word rows: at most four column pieces.
struct Digit4 {
  int nterm;
  int tcol[4], tshr[4], tshl[4];
  uint32_t tmask[4], txr[4];
};

__device__ __forceinline__ uint32_t digit_of4(int4 r, const Digit4 &ks) {
  uint32_t v = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t >= ks.nterm) break;
    const int c = ks.tcol[t];
    const uint32_t col = (uint32_t)(c == 0 ? r.x : c == 1 ? r.y : c == 2 ? r.z : r.w) ^ ks.txr[t];
    v |= ((col >> ks.tshr[t]) & ks.tmask[t]) << ks.tshl[t];
  }
  return v;
}

__global__ void __launch_bounds__(kSortThreads)
k_hist(const int32_t *__restrict__ rows, int64_t nrows, int width, int64_t per_block,
       KeySpec ks, uint32_t *__restrict__ hist, int grid) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t lo = (int64_t)blockIdx.x * per_block;
  int64_t hi = min(nrows, lo + per_block);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&h[digit_of(rows + i * width, ks)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * grid + blockIdx.x] = h[d];
}

// Digit counts of rows [lo, hi) into h (shared memory), eight independent
// 16-byte loads in flight per thread.
template <class Spec>
__device__ __forceinline__ void hist4_range(const int4 *__restrict__ rows, int64_t lo, int64_t hi, const Spec &ks,
                                            uint32_t *h) {
  const int64_t step = blockDim.x;
  int64_t i = lo + threadIdx.x;
  for (; i + 7 * step < hi; i += 8 * step) {
    int4 r[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) r[t] = __ldcg(rows + i + t * step);
#pragma unroll
    for (int t = 0; t < 8; ++t) atomicAdd(&h[digit_of4(r[t], ks)], 1u);
  }
  for (; i < hi; i += step) atomicAdd(&h[digit_of4(__ldcg(rows + i), ks)], 1u);
}

// The same histogram over four-word rows read as int4 (16-byte aligned rows).
__global__ void __launch_bounds__(kSortThreads)
k_hist4(const int4 *__restrict__ rows, int64_t nrows, int64_t per_block, KeySpec ks,
        uint32_t *__restrict__ hist, int grid) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t lo = (int64_t)blockIdx.x * per_block;
  int64_t hi = min(nrows, lo + per_block);
  hist4_range(rows, lo, hi, ks, h);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * grid + blockIdx.x] = h[d];
}

// Exclusive scan of `len` uint32 values in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(uint32_t *__restrict__ a, int64_t len) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < len; base += 1024) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < len ? a[i] : 0;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    uint32_t before = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
    if (i < len) a[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[31];
    __syncthreads();
  }
}

template <int W>
__global__ void __launch_bounds__(kSortThreads)
k_scatter(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t nrows,
          int64_t per_block, KeySpec ks, const uint32_t *__restrict__ starts, int grid) {
  __shared__ uint32_t s_base[kRadix];
  __shared__ uint32_t s_cnt[kSortWarps][kRadix];
  __shared__ uint32_t s_tile[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    s_base[d] = starts[(int64_t)d * grid + blockIdx.x];
  int64_t lo = (int64_t)blockIdx.x * per_block;
  int64_t hi = min(nrows, lo + per_block);
  const uint32_t lt = lanemask_lt();
  for (int64_t tile = lo; tile < hi; tile += kTile) {
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t dig[kItems], rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      int64_t i = tile + (int64_t)warp * 32 * kItems + r * 32 + lane;
      bool valid = i < hi;
      uint32_t d = valid ? digit_of(in + i * W, ks) : kRadix;
      uint32_t peers = __match_any_sync(0xffffffffu, d);
      int leader = __ffs(peers) - 1;
      uint32_t prev = 0;
      if (valid && lane == leader) {
        prev = s_cnt[warp][d];
        s_cnt[warp][d] = prev + __popc(peers);
      }
      prev = __shfl_sync(0xffffffffu, prev, leader);
      dig[r] = d;
      rank[r] = prev + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t t = s_cnt[w][d];
        s_cnt[w][d] = acc;
        acc += t;
      }
      s_tile[d] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      int64_t i = tile + (int64_t)warp * 32 * kItems + r * 32 + lane;
      if (i < hi) {
        uint32_t d = dig[r];
        int64_t pos = (int64_t)s_base[d] + s_cnt[warp][d] + rank[r];
        const int32_t *src = in + i * W;
        int32_t *dst = out + pos * W;
#pragma unroll
        for (int w = 0; w < W; ++w) dst[w] = src[w];
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) s_base[d] += s_tile[d];
    __syncthreads();
  }
}

// The same pass for four-word rows (the arc rows of the graph build and the
// matches of 4-vertex patterns), with coalesced writes: each row is loaded
// once as an int4, the tile is reordered by digit in shared memory, and the
// tile's run of each digit is written out by consecutive threads.

// Shared memory of one block's reorder-then-write pass over four-word rows.
struct Scatter4Smem {
  uint32_t base[2][kRadix];                // global start of each digit for this block's current
                                           // tile and for the next one (alternating)
  __align__(16) uint16_t cnt[kSortWarps][kRadix];  // per-warp digit counts, then warp offsets
  __align__(8) uint16_t first[kRadix];     // tile-local start of each digit
  int4 rows[kTile];                        // the tile in digit order
  uint16_t dig[kTile];                     // digit of each reordered row
  uint32_t wsum[kSortWarps];
};

// Rows [lo, hi) of `in` to their places in `out`; sm.base holds the block's
// global start of each digit (written before the call by the whole block).
template <class Spec>
__device__ __forceinline__ void scatter4_range(const int4 *__restrict__ in, int4 *__restrict__ out, int64_t lo,
                                               int64_t hi, const Spec &ks, Scatter4Smem &sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  // each tile's rows are loaded while the previous tile is being reordered
  int4 next[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = lo + warp * 32 * kItems + r * 32 + lane;
    next[r] = i < hi ? __ldcg(in + i) : make_int4(0, 0, 0, 0);
  }
  for (int i = threadIdx.x; i < kSortWarps * kRadix / 8; i += blockDim.x)
    reinterpret_cast<uint4 *>(&sm.cnt[0][0])[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  int cur = 0;  // sm.base[cur]: this tile's digit starts (the caller filled sm.base[0])
  for (int64_t tile = lo; tile < hi; tile += kTile) {
    const int tn = (int)min((int64_t)kTile, hi - tile);
    int4 row[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      row[r] = next[r];
      const int64_t i = tile + kTile + warp * 32 * kItems + r * 32 + lane;
      next[r] = i < hi ? __ldcg(in + i) : make_int4(0, 0, 0, 0);
    }
    uint32_t dig[kItems], rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int li = warp * 32 * kItems + r * 32 + lane;
      const bool valid = li < tn;
      const uint32_t d = valid ? digit_of4(row[r], ks) : kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t prev = 0;
      if (valid && lane == leader) {
        prev = sm.cnt[warp][d];
        sm.cnt[warp][d] = (uint16_t)(prev + __popc(peers));
      }
      prev = __shfl_sync(0xffffffffu, prev, leader);
      dig[r] = d;
      rank[r] = prev + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets (in place), the tile-local start and the next
    // tile's global start; each thread owns four consecutive digits, whose
    // 16-bit counters it moves as one 64-bit word (a tile holds at most 1024
    // rows, so no 16-bit lane of a sum carries into the next)
    {
      static_assert(kRadix == 4 * kSortThreads, "four digits per thread");
      const int d0 = threadIdx.x * 4;
      uint64_t acc = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        uint64_t *c = reinterpret_cast<uint64_t *>(&sm.cnt[w][d0]);
        const uint64_t t = *c;
        *c = acc;
        acc += t;
      }
      const uint32_t v0 = (uint32_t)(acc & 0xffff), v1 = (uint32_t)((acc >> 16) & 0xffff),
                     v2 = (uint32_t)((acc >> 32) & 0xffff), v3 = (uint32_t)(acc >> 48);
      const uint32_t sum = v0 + v1 + v2 + v3;
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) sm.wsum[warp] = x;
      __syncthreads();
      uint32_t before = x - sum;
      for (int w = 0; w < warp; ++w) before += sm.wsum[w];
      const uint64_t f0 = before, f1 = before + v0, f2 = f1 + v1, f3 = f2 + v2;
      *reinterpret_cast<uint64_t *>(&sm.first[d0]) = f0 | (f1 << 16) | (f2 << 32) | (f3 << 48);
      const uint4 b = *reinterpret_cast<const uint4 *>(&sm.base[cur][d0]);
      *reinterpret_cast<uint4 *>(&sm.base[cur ^ 1][d0]) = make_uint4(b.x + v0, b.y + v1, b.z + v2, b.w + v3);
    }
    __syncthreads();
    // reorder the tile by digit in shared memory
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int li = warp * 32 * kItems + r * 32 + lane;
      if (li < tn) {
        const uint32_t d = dig[r];
        const int lp = sm.first[d] + sm.cnt[warp][d] + rank[r];
        sm.rows[lp] = row[r];
        sm.dig[lp] = (uint16_t)d;
      }
    }
    __syncthreads();
    // consecutive threads write consecutive rows of each digit's run; the
    // counters are cleared for the next tile meanwhile
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
      const uint32_t d = sm.dig[t];
      out[(int64_t)sm.base[cur][d] + (t - sm.first[d])] = sm.rows[t];
    }
    for (int i = threadIdx.x; i < kSortWarps * kRadix / 8; i += blockDim.x)
      reinterpret_cast<uint4 *>(&sm.cnt[0][0])[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    cur ^= 1;
  }
}

__global__ void __launch_bounds__(kSortThreads)
k_scatter4(const int4 *__restrict__ in, int4 *__restrict__ out, int64_t nrows, int64_t per_block, KeySpec ks,
           const uint32_t *__restrict__ starts, int grid) {
  __shared__ Scatter4Smem sm;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    sm.base[0][d] = starts[(int64_t)d * grid + blockIdx.x];
  const int64_t lo = (int64_t)blockIdx.x * per_block;
  scatter4_range(in, out, lo, min(nrows, lo + per_block), ks, sm);
}

// The same reorder-then-write pass for rows of W words (2..8), staged as
// plain words: tiles of 1,024 rows up to four words, 512 rows above.
template <int W>
__global__ void __launch_bounds__(kSortThreads)
k_scatter_staged(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t nrows, int64_t per_block,
                 KeySpec ks, const uint32_t *__restrict__ starts, int grid) {
  constexpr int kIt = W <= 4 ? kItems : kItems / 2;
  constexpr int kT = kSortThreads * kIt;
  __shared__ uint32_t s_base[kRadix];
  __shared__ uint16_t s_cnt[kSortWarps][kRadix];
  __shared__ uint16_t s_first[kRadix];
  __shared__ uint16_t s_num[kRadix];
  __shared__ int32_t s_rows[kT * W];
  __shared__ uint16_t s_dig[kT];
  __shared__ uint32_t s_wsum[kSortWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    s_base[d] = starts[(int64_t)d * grid + blockIdx.x];
  const int64_t lo = (int64_t)blockIdx.x * per_block;
  const int64_t hi = min(nrows, lo + per_block);
  const uint32_t lt = lanemask_lt();
  for (int64_t tile = lo; tile < hi; tile += kT) {
    const int tn = (int)min((int64_t)kT, hi - tile);
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += blockDim.x) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t dig[kIt], rank[kIt];
#pragma unroll
    for (int r = 0; r < kIt; ++r) {
      const int li = warp * 32 * kIt + r * 32 + lane;
      const bool valid = li < tn;
      const uint32_t d = valid ? digit_of(in + (tile + li) * W, ks) : kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t prev = 0;
      if (valid && lane == leader) {
        prev = s_cnt[warp][d];
        s_cnt[warp][d] = (uint16_t)(prev + __popc(peers));
      }
      prev = __shfl_sync(0xffffffffu, prev, leader);
      dig[r] = d;
      rank[r] = prev + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t t = s_cnt[w][d];
        s_cnt[w][d] = (uint16_t)acc;
        acc += t;
      }
      s_num[d] = (uint16_t)acc;
    }
    __syncthreads();
    {
      constexpr int kPer = kRadix / kSortThreads;
      uint32_t v[kPer], sum = 0;
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        v[t] = s_num[threadIdx.x * kPer + t];
        sum += v[t];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[warp] = x;
      __syncthreads();
      uint32_t before = x - sum;
      for (int w = 0; w < warp; ++w) before += s_wsum[w];
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        s_first[threadIdx.x * kPer + t] = (uint16_t)before;
        before += v[t];
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kIt; ++r) {
      const int li = warp * 32 * kIt + r * 32 + lane;
      if (li < tn) {
        const uint32_t d = dig[r];
        const int lp = s_first[d] + s_cnt[warp][d] + rank[r];
        const int32_t *src = in + (tile + li) * W;
#pragma unroll
        for (int w = 0; w < W; ++w) s_rows[lp * W + w] = src[w];
        s_dig[lp] = (uint16_t)d;
      }
    }
    __syncthreads();
    // word by word, so consecutive threads write consecutive words of each run
    for (int e = threadIdx.x; e < tn * W; e += blockDim.x) {
      const int t = e / W, w = e - t * W;
      const uint32_t d = s_dig[t];
      out[((int64_t)s_base[d] + (t - s_first[d])) * W + w] = s_rows[e];
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) s_base[d] += s_num[d];
    __syncthreads();
  }
}

template <int W>
void launch_scatter(const int32_t *in, int32_t *out, int64_t nrows, int64_t per_block, KeySpec ks,
                    const uint32_t *starts, int grid, cudaStream_t s) {
  // int4 rows need 16-byte aligned buffers (a caller's output buffer may not be)
  const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
  if (W == 4 && aligned)
    k_scatter4<<<grid, kSortThreads, 0, s>>>(reinterpret_cast<const int4 *>(in), reinterpret_cast<int4 *>(out),
                                             nrows, per_block, ks, starts, grid);
  else if constexpr (W >= 2 && W <= 8)
    k_scatter_staged<W><<<grid, kSortThreads, 0, s>>>(in, out, nrows, per_block, ks, starts, grid);
  else
    k_scatter<W><<<grid, kSortThreads, 0, s>>>(in, out, nrows, per_block, ks, starts, grid);
}

using ScatterFn = void (*)(const int32_t *, int32_t *, int64_t, int64_t, KeySpec,
                           const uint32_t *, int, cudaStream_t);

ScatterFn scatter_for(int width) {
  switch (width) {
    case 1: return launch_scatter<1>;
    case 2: return launch_scatter<2>;
    case 3: return launch_scatter<3>;
    case 4: return launch_scatter<4>;
    case 5: return launch_scatter<5>;
    case 6: return launch_scatter<6>;
    case 7: return launch_scatter<7>;
    case 8: return launch_scatter<8>;
    case 9: return launch_scatter<9>;
    case 10: return launch_scatter<10>;
    case 11: return launch_scatter<11>;
    case 12: return launch_scatter<12>;
    case 13: return launch_scatter<13>;
    case 14: return launch_scatter<14>;
    case 15: return launch_scatter<15>;
    case 16: return launch_scatter<16>;
    case 17: return launch_scatter<17>;
    case 18: return launch_scatter<18>;
    case 19: return launch_scatter<19>;
    case 20: return launch_scatter<20>;
    case 21: return launch_scatter<21>;
    default: return nullptr;
  }
}


constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
  __shared__ uint32_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kScanThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = s;
  }
  __syncthreads();
  uint32_t before = (warp ? ws[warp - 1] : 0) + x - v;
  *total = ws[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

// ---- all passes in one cooperative launch (four-word rows) ------------------
//
// Every block of the grid is resident (cooperative launch), so the three
// phases of a pass -- per-block histogram, per-digit prefix over blocks,
// reorder-then-write -- are separated by grid-wide barriers instead of
// kernel boundaries.  Data that other blocks wrote is read through L2
// (__ldcg).  A barrier waits at most kBarrierNs (long enough for blocks that
// wait for SMs held by kernels of other streams); a block that gives up sets
// *err and returns, and every other block returns at its next barrier, so
// the launch always ends (the host then reports an error).
constexpr int kMaxSortPasses = (4 * 32 + kDigitBits - 1) / kDigitBits;
constexpr uint64_t kBarrierNs = 10ull * 1000 * 1000 * 1000;
constexpr int kWarpScanBelow = 128;  // grids smaller than this scan one digit per warp
// The fused sort waits for its barrier status before it returns; below this
// many rows that wait costs more than the launches it saves, and the sort
// runs as separate kernels that the caller's next launches can queue behind.
constexpr int64_t kFusedMinRows = 1 << 18;

struct FusedSort4 {
  int4 *a, *b;                 // pass p reads a (p even) or b and writes the other
  int64_t nrows, per_block;
  int grid, passes;
  uint32_t *hist;              // [kRadix * grid] per-block digit counts
  uint32_t *part;              // [kRadix * grid] counts of the same digit in earlier blocks
  uint32_t *tot;               // [kRadix] digit totals
  unsigned int *bar;           // arrivals (zero at launch)
  int *err;                    // set when a barrier gave up
  Digit4 ks[kMaxSortPasses];
};

__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int target, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
      if (*(volatile unsigned int *)bar >= target) break;
      if (globaltimer_ns() - t0 > kBarrierNs) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    if (*(volatile int *)err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kSortThreads, 3) k_sort4_fused(const __grid_constant__ FusedSort4 F) {
  __shared__ Scatter4Smem sm;
  const int b = blockIdx.x, grid = F.grid;
  const int64_t lo = (int64_t)b * F.per_block;
  const int64_t hi = min(F.nrows, lo + F.per_block);
  unsigned int target = 0;
  for (int p = 0; p < F.passes; ++p) {
    const int4 *in = (p & 1) ? F.b : F.a;
    int4 *out = (p & 1) ? F.a : F.b;
    const Digit4 &ks = F.ks[p];
    // 1. this block's digit counts
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) sm.base[0][d] = 0;
    __syncthreads();
    hist4_range(in, lo, hi, ks, sm.base[0]);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) F.hist[(int64_t)d * grid + b] = sm.base[0][d];
    target += grid;
    if (!grid_barrier(F.bar, target, F.err)) return;
    // 2. each digit's counts in earlier blocks, and its total: on a large
    //    grid one block per digit (a block-wide scan per 256 blocks); on a
    //    small one, where that would leave few blocks scanning many digits
    //    one after another, one warp per digit
    if (grid >= kWarpScanBelow) {
      // each thread takes up to four consecutive blocks' counts, so one
      // block-wide scan covers a grid of up to 1,024 blocks
      const int per = (grid + kSortThreads - 1) / kSortThreads;
      for (int d = b; d < kRadix; d += grid) {
        const uint32_t *h = F.hist + (int64_t)d * grid;
        uint32_t *q = F.part + (int64_t)d * grid;
        if (per <= 4) {
          const int c0 = threadIdx.x * per;
          uint32_t v[4] = {0u, 0u, 0u, 0u}, sum = 0;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (t < per && c0 + t < grid) {
              v[t] = __ldcg(h + c0 + t);
              sum += v[t];
            }
          uint32_t all;
          uint32_t run = block_excl_scan(sum, &all);
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (t < per && c0 + t < grid) {
              q[c0 + t] = run;
              run += v[t];
            }
          if (threadIdx.x == 0) F.tot[d] = all;
        } else {
          uint32_t run = 0;
          for (int c0 = 0; c0 < grid; c0 += blockDim.x) {
            const int c = c0 + threadIdx.x;
            const uint32_t v = c < grid ? __ldcg(h + c) : 0u;
            uint32_t chunk;
            const uint32_t before = block_excl_scan(v, &chunk);
            if (c < grid) q[c] = run + before;
            run += chunk;
          }
          if (threadIdx.x == 0) F.tot[d] = run;
        }
      }
    } else {
      const int lane = threadIdx.x & 31, nw = grid * kSortWarps;
      for (int d = b * kSortWarps + (threadIdx.x >> 5); d < kRadix; d += nw) {
        const uint32_t *h = F.hist + (int64_t)d * grid;
        uint32_t *q = F.part + (int64_t)d * grid;
        uint32_t run = 0;
        for (int c0 = 0; c0 < grid; c0 += 32) {
          const int c = c0 + lane;
          const uint32_t v = c < grid ? __ldcg(h + c) : 0u;
          uint32_t x = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
          }
          if (c < grid) q[c] = run + x - v;
          run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) F.tot[d] = run;
      }
    }
    target += grid;
    if (!grid_barrier(F.bar, target, F.err)) return;
    // 3. global start of each digit for this block, then reorder and write
    {
      constexpr int kPer = kRadix / kSortThreads;
      uint32_t v[kPer], sum = 0;
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        v[t] = __ldcg(F.tot + threadIdx.x * kPer + t);
        sum += v[t];
      }
      uint32_t all;
      uint32_t before = block_excl_scan(sum, &all);
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int d = threadIdx.x * kPer + t;
        sm.base[0][d] = before + __ldcg(F.part + (int64_t)d * grid + b);
        before += v[t];
      }
    }
    __syncthreads();
    scatter4_range(in, out, lo, hi, ks, sm);
    if (p + 1 == F.passes) break;
    target += grid;
    if (!grid_barrier(F.bar, target, F.err)) return;
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_tile_sums(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  uint32_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_tile_scan(const uint32_t *__restrict__ in, int64_t n, const uint32_t *__restrict__ offs,
            uint32_t *__restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(s, &total) + offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

}  // namespace

hm_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return HM_OK;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  uint32_t *sums = nullptr;
  HM_CUDA_TRY(cudaMallocAsync(&sums, sizeof(uint32_t) * (size_t)tiles, s));
  k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  k_scan<<<1, 1024, 0, s>>>(sums, tiles);
  k_tile_scan<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out);
  HM_CUDA_TRY(cudaFreeAsync(sums, s));
  HM_CUDA_TRY(cudaGetLastError());
  return HM_OK;
}



int bits_for(int64_t n) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < n) ++b;
  return b;
}

int num_sms() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_relaxed);
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 1;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

hm_status radix_sort_rows(int32_t *rows, int32_t *tmp, int64_t nrows, int width,
                          const int *key_cols, int nkey, int bits, cudaStream_t stream, int *launches) {
  int b[kMaxKeyCols];
  uint32_t x[kMaxKeyCols];
  if (nkey < 1 || nkey > kMaxKeyCols) return HM_ERR_ARG;
  for (int i = 0; i < nkey; ++i) {
    b[i] = bits;
    x[i] = 0;
  }
  return radix_sort_rows_cols(rows, tmp, nrows, width, key_cols, b, x, nkey, stream, launches);
}

// All passes of a sort of 16-byte aligned four-word rows in one cooperative
// launch.  *ran is false (and nothing was launched) when the device cannot
// hold a grid of resident blocks for it; the caller then runs the passes as
// separate kernels.
static hm_status sort4_fused(int32_t *rows, int32_t *tmp, int64_t nrows, KeySpec ks, int passes,
                             cudaStream_t stream, bool *ran) {
  *ran = false;
  static std::atomic<int> per_sm{-1};
  int nb = per_sm.load(std::memory_order_relaxed);
  if (nb < 0) {
    int coop = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sort4_fused, kSortThreads, 0) != cudaSuccess)
      nb = 0;
    cudaGetLastError();
    per_sm.store(nb, std::memory_order_relaxed);
  }
  if (nb <= 0 || passes > kMaxSortPasses) return HM_OK;
  int grid = (int)std::min<int64_t>((nrows + kTile - 1) / kTile, (int64_t)num_sms() * nb);
  int64_t per_block = (nrows + grid - 1) / grid;
  per_block = (per_block + kTile - 1) / kTile * kTile;
  grid = (int)((nrows + per_block - 1) / per_block);
  const int64_t nhist = (int64_t)kRadix * grid;
  uint32_t *buf = nullptr;
  HM_CUDA_TRY(cudaMallocAsync(&buf, sizeof(uint32_t) * (size_t)(2 * nhist + kRadix + 4), stream));
  FusedSort4 F{};
  F.a = reinterpret_cast<int4 *>(rows);
  F.b = reinterpret_cast<int4 *>(tmp);
  F.nrows = nrows;
  F.per_block = per_block;
  F.grid = grid;
  F.passes = passes;
  F.hist = buf;
  F.part = buf + nhist;
  F.tot = buf + 2 * nhist;
  F.bar = reinterpret_cast<unsigned int *>(buf + 2 * nhist + kRadix);
  F.err = reinterpret_cast<int *>(buf + 2 * nhist + kRadix + 1);
  for (int p = 0; p < passes; ++p) {
    set_pass(ks, p * kDigitBits);
    Digit4 &d = F.ks[p];
    d.nterm = ks.nterm;
    for (int t = 0; t < ks.nterm; ++t) {
      d.tcol[t] = ks.tcol[t];
      d.tshr[t] = ks.tshr[t];
      d.tshl[t] = ks.tshl[t];
      d.tmask[t] = ks.tmask[t];
      d.txr[t] = ks.txr[t];
    }
  }
  HM_CUDA_TRY(cudaMemsetAsync(F.bar, 0, 2 * sizeof(uint32_t), stream));
  void *args[] = {&F};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_sort4_fused, dim3(grid), dim3(kSortThreads),
                                                    args, 0, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not launched: the caller takes the multi-kernel path
    HM_CUDA_TRY(cudaFreeAsync(buf, stream));
    return HM_OK;
  }
  *ran = true;
  if (passes & 1)
    HM_CUDA_TRY(cudaMemcpyAsync(rows, tmp, sizeof(int4) * (size_t)nrows, cudaMemcpyDeviceToDevice, stream));
  int err = 0;
  HM_CUDA_TRY(cudaMemcpyAsync(&err, F.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  HM_CUDA_TRY(cudaFreeAsync(buf, stream));
  HM_CUDA_TRY(cudaStreamSynchronize(stream));
  return err ? HM_ERR_CUDA : HM_OK;
}

hm_status radix_sort_rows_cols(int32_t *rows, int32_t *tmp, int64_t nrows, int width,
                               const int *key_cols, const int *key_bits, const uint32_t *key_xor,
                               int nkey, cudaStream_t stream, int *launches) {
  if (nrows <= 1) return HM_OK;
  ScatterFn scatter = scatter_for(width);
  if (!scatter || nkey < 1 || nkey > kMaxKeyCols) return HM_ERR_ARG;
  KeySpec ks{};
  ks.ncols = nkey;
  int total_bits = 0;
  for (int i = 0; i < nkey; ++i) {
    if (key_bits[i] < 1 || key_bits[i] > 32 || key_cols[i] < 0 || key_cols[i] >= width)
      return HM_ERR_ARG;
    ks.cols[i] = key_cols[i];
    ks.bits[i] = key_bits[i];
    ks.xr[i] = key_xor[i];
    total_bits += key_bits[i];
  }
  const int passes = (total_bits + kDigitBits - 1) / kDigitBits;
  if (launches) *launches = 5 * passes;
  if (width == 4 && nrows >= kFusedMinRows &&
      (((reinterpret_cast<uintptr_t>(rows) | reinterpret_cast<uintptr_t>(tmp)) & 15u) == 0)) {
    bool ran = false;
    const hm_status fs = sort4_fused(rows, tmp, nrows, ks, passes, stream, &ran);
    if (fs != HM_OK) return fs;
    if (ran) {
      if (launches) *launches = 1;
      return HM_OK;
    }
  }
  int grid = (int)std::min<int64_t>((nrows + kTile - 1) / kTile, (int64_t)num_sms() * 4);
  int64_t per_block = (nrows + grid - 1) / grid;
  per_block = (per_block + kTile - 1) / kTile * kTile;
  grid = (int)((nrows + per_block - 1) / per_block);
  uint32_t *hist = nullptr;
  const int64_t nhist = (int64_t)kRadix * grid;
  const int64_t tiles = (nhist + kScanTile - 1) / kScanTile;
  HM_CUDA_TRY(cudaMallocAsync(&hist, sizeof(uint32_t) * (size_t)(2 * nhist + tiles), stream));
  uint32_t *starts = hist + nhist, *sums = starts + nhist;
  int32_t *a = rows, *b = tmp;
  for (int p = 0; p < passes; ++p) {
    set_pass(ks, p * kDigitBits);
    if (width == 4 && ((reinterpret_cast<uintptr_t>(a) & 15u) == 0))
      k_hist4<<<grid, kSortThreads, 0, stream>>>(reinterpret_cast<const int4 *>(a), nrows, per_block, ks, hist,
                                                 grid);
    else
      k_hist<<<grid, kSortThreads, 0, stream>>>(a, nrows, width, per_block, ks, hist, grid);
    // exclusive scan of the (digit, block) counts over many blocks
    k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, stream>>>(hist, nhist, sums);
    k_scan<<<1, 1024, 0, stream>>>(sums, tiles);
    k_tile_scan<<<(unsigned)tiles, kScanThreads, 0, stream>>>(hist, nhist, sums, starts);
    scatter(a, b, nrows, per_block, ks, starts, grid, stream);
    std::swap(a, b);
  }
  if (a != rows)
    HM_CUDA_TRY(cudaMemcpyAsync(rows, a, sizeof(int32_t) * nrows * width,
                                cudaMemcpyDeviceToDevice, stream));
  HM_CUDA_TRY(cudaFreeAsync(hist, stream));
  HM_CUDA_TRY(cudaGetLastError());
  return HM_OK;
}

}  // namespace hm
