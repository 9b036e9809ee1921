// Tree construction on sm_103a (Section 4.3 of the paper): root cell, Morton
// keys, stable LSD radix sort, reorder into Morton order, octree link and
// bottom-up moments, i-groups.
//
// FP64 arithmetic that decides an integer or feeds the opening criterion
// (key scaling, moment sums, centres) is written with explicit _rn
// intrinsics so that no multiply-add is contracted: the results are the
// IEEE results of the operation sequence stated in each kernel.
#include <cfloat>
#include <utility>
#include <vector>

#include "afd_internal.cuh"
#include "afd_split.cuh"

namespace afd {
namespace {

constexpr int kThreads = 256;
#ifndef AFD_MAX_SIDX
#define AFD_MAX_SIDX 2u  // largest log2 of the j-stream split of a remainder unit
#endif

inline unsigned blocks_for(int64_t n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

// ---------------------------------------------------------------------------
// Root cell: bounding box of all particles, centre (min+max)/2, side L = the
// smallest power of two >= 1.000001 * largest extent (1 for a zero extent).
// One pass; the last block to finish reduces the per-block partials.
// ---------------------------------------------------------------------------
constexpr int kRootBlocks = 608;

__global__ void __launch_bounds__(kThreads) k_root(const double *__restrict__ x,
                                                   const double *__restrict__ y,
                                                   const double *__restrict__ z,
                                                   const double *__restrict__ m, int64_t n,
                                                   unsigned long long *__restrict__ part,
                                                   unsigned *__restrict__ counter,
                                                   double *__restrict__ root, int *status) {
  unsigned long long klo[3] = {~0ull, ~0ull, ~0ull}, khi[3] = {0ull, 0ull, 0ull};
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v[3] = {x[i], y[i], z[i]};
    const double mv = m[i];
    bad |= !isfinite(mv);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      bad |= !isfinite(v[d]);
      box_keys(v[d], klo[d], khi[d]);
    }
  }
  __shared__ unsigned long long sh[kThreads / 32][6];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    klo[d] = warp_min_key(klo[d]);
    khi[d] = warp_max_key(khi[d]);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStNonFinite);
  if (lane == 0)
    for (int d = 0; d < 3; d++) {
      sh[warp][d] = klo[d];
      sh[warp][3 + d] = khi[d];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b[6];
    for (int d = 0; d < 6; d++) b[d] = sh[0][d];
    for (int w = 1; w < kThreads / 32; w++)
      for (int d = 0; d < 3; d++) {
        b[d] = min(b[d], sh[w][d]);
        b[3 + d] = max(b[3 + d], sh[w][3 + d]);
      }
    for (int d = 0; d < 6; d++) part[blockIdx.x * 6 + d] = b[d];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block reduces all partials, every thread a strided share
  for (int d = 0; d < 3; d++) {
    klo[d] = ~0ull;
    khi[d] = 0ull;
  }
  for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x)
    for (int d = 0; d < 3; d++) {
      klo[d] = min(klo[d], __ldcg(&part[k * 6 + d]));
      khi[d] = max(khi[d], __ldcg(&part[k * 6 + 3 + d]));
    }
  for (int d = 0; d < 3; d++) {
    klo[d] = warp_min_key(klo[d]);
    khi[d] = warp_max_key(khi[d]);
  }
  __syncthreads();
  if (lane == 0)
    for (int d = 0; d < 3; d++) {
      sh[warp][d] = klo[d];
      sh[warp][3 + d] = khi[d];
    }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned long long b[6];
  for (int d = 0; d < 6; d++) b[d] = sh[0][d];
  for (int w = 1; w < kThreads / 32; w++)
    for (int d = 0; d < 3; d++) {
      b[d] = min(b[d], sh[w][d]);
      b[3 + d] = max(b[3 + d], sh[w][3 + d]);
    }
  if (!root_from_keys(b, b + 3, root)) atomicOr(status, kStNonFinite);
  *counter = 0u;  // ready for the next launch
}

// Root cells of several systems: block b reduces tile b (a particle range
// inside one system) to partials; then one block per system reduces its
// tiles. Same root rule as k_root.
constexpr int kRootTile = 8192;

__global__ void __launch_bounds__(kThreads) k_root_tiles(const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ m,
                                                         const int4 *__restrict__ tiles,
                                                         unsigned long long *__restrict__ part,
                                                         int *status) {
  const int4 t = tiles[blockIdx.x];
  unsigned long long klo[3] = {~0ull, ~0ull, ~0ull}, khi[3] = {0ull, 0ull, 0ull};
  int bad = 0;
  for (int64_t i = (int64_t)t.y + threadIdx.x; i < (int64_t)t.z; i += blockDim.x) {
    const double v[3] = {x[i], y[i], z[i]};
    bad |= !isfinite(m[i]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      bad |= !isfinite(v[d]);
      box_keys(v[d], klo[d], khi[d]);
    }
  }
  __shared__ unsigned long long sh[kThreads / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    klo[d] = warp_min_key(klo[d]);
    khi[d] = warp_max_key(khi[d]);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStNonFinite);
  if (lane == 0)
    for (int d = 0; d < 3; d++) {
      sh[warp][d] = klo[d];
      sh[warp][3 + d] = khi[d];
    }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned long long b[6];
  for (int d = 0; d < 6; d++) b[d] = sh[0][d];
  for (int w = 1; w < kThreads / 32; w++)
    for (int d = 0; d < 3; d++) {
      b[d] = min(b[d], sh[w][d]);
      b[3 + d] = max(b[3 + d], sh[w][3 + d]);
    }
  for (int d = 0; d < 6; d++) part[(size_t)blockIdx.x * 6 + d] = b[d];
}

__global__ void __launch_bounds__(kThreads) k_root_final(const unsigned long long *__restrict__ part,
                                                         const int *__restrict__ tile_first,
                                                         double *__restrict__ root, int *status) {
  const int sys = blockIdx.x;
  const int t0 = tile_first[sys], t1 = tile_first[sys + 1];
  unsigned long long klo[3] = {~0ull, ~0ull, ~0ull}, khi[3] = {0ull, 0ull, 0ull};
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
    for (int d = 0; d < 3; d++) {
      klo[d] = min(klo[d], part[(size_t)t * 6 + d]);
      khi[d] = max(khi[d], part[(size_t)t * 6 + 3 + d]);
    }
  __shared__ unsigned long long sh[kThreads / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < 3; d++) {
    klo[d] = warp_min_key(klo[d]);
    khi[d] = warp_max_key(khi[d]);
  }
  if (lane == 0)
    for (int d = 0; d < 3; d++) {
      sh[warp][d] = klo[d];
      sh[warp][3 + d] = khi[d];
    }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* r = root + 4 * (size_t)sys;
  if (t1 == t0) {  // empty system
    r[0] = r[1] = r[2] = 0.0;
    r[3] = 1.0;
    return;
  }
  unsigned long long b[6];
  for (int d = 0; d < 6; d++) b[d] = sh[0][d];
  for (int w = 1; w < kThreads / 32; w++)
    for (int d = 0; d < 3; d++) {
      b[d] = min(b[d], sh[w][d]);
      b[3 + d] = max(b[3 + d], sh[w][3 + d]);
    }
  if (!root_from_keys(b, b + 3, r)) atomicOr(status, kStNonFinite);
}

// System of each particle (caller order) from the system offsets.
__global__ void __launch_bounds__(kThreads) k_sys_of(const int64_t *__restrict__ sys_off, int n_sys,
                                                     int64_t n, uint32_t *__restrict__ sys_of) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_sys;  // last s with sys_off[s] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sys_off[mid] <= i) lo = mid;
    else hi = mid;
  }
  sys_of[i] = (uint32_t)lo;
}

// ---------------------------------------------------------------------------
// Morton keys: q_d = clamp(floor((x_d - (c_d - L/2)) * 2^21 / L)), bits
// interleaved x-y-z from the most significant end (63 bits used).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// clamp(floor((v - corner) * 2^s), 0, 2^21 - 1) with 2^s = 2^21 / L (L a
// power of two, so the product is exact unless it underflows, and then it
// is below 1): the difference in FP64, its integer part from its exponent
// and mantissa on the integer pipes (GB300's FP64 rate is low).
__device__ __forceinline__ uint32_t grid_coord(double v, double corner, int s) {
  const double d = __dsub_rn(v, corner);
  if (!(d > 0.0)) return 0u;
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e == 0) return 0u;          // subnormal: the product is below 1
  const int k = e - 1023 + s;     // d * 2^s = 1.m x 2^k
  if (k < 0) return 0u;
  if (k >= 21) return 2097151u;
  const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
  return (uint32_t)(mant >> (52 - k));
}

__global__ void __launch_bounds__(kThreads) k_keys(const double *__restrict__ x,
                                                   const double *__restrict__ y,
                                                   const double *__restrict__ z, int64_t n,
                                                   const double *__restrict__ roots,
                                                   const uint32_t *__restrict__ sys_of,
                                                   uint64_t *__restrict__ keys,
                                                   uint32_t *__restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *root = roots + (sys_of ? 4 * (size_t)sys_of[i] : 0);
  const double L = root[3];
  const double half = __dmul_rn(L, 0.5);
  // 2^21 / L = 2^s: L = 2^(e_L - 1023)
  const int s = 1044 - (int)(((unsigned long long)__double_as_longlong(L) >> 52) & 0x7ffu);
  const uint32_t qx = grid_coord(x[i], __dsub_rn(root[0], half), s);
  const uint32_t qy = grid_coord(y[i], __dsub_rn(root[1], half), s);
  const uint32_t qz = grid_coord(z[i], __dsub_rn(root[2], half), s);
  keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
  perm[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, index), 8-bit digits, 8 passes (Section 6.2
// sorts with 8-bit chunks). One launch counts the digits of every pass;
// then each pass is one launch: tiles of kSortTile keys, taken in input
// order from a counter, count their digits, publish the counts, and find
// each digit's offset among the preceding tiles by decoupled look-back
// (a tile adds its predecessors' published counts back to the first
// inclusive prefix it meets), then scatter their keys stably: each tile
// reads its keys once, ranks them in input order (warp match for the lanes
// of a round, warp-private counters for the rounds, offsets over the warps
// per digit), places them in sorted order in shared memory and writes them
// out in runs of equal digits.
// ---------------------------------------------------------------------------
#ifndef AFD_SORT_ROUNDS
#define AFD_SORT_ROUNDS 16  // rounds of 256 keys per sort tile
#endif
constexpr int kSortThreads = 256;
constexpr int kSortRounds = AFD_SORT_ROUNDS;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortMaxPasses = 10;  // 8 key bytes + up to 2 bytes of system id
// look-back words: the count (or inclusive prefix) in bits 0-29, the state
// in bits 30-31
constexpr uint32_t kLookAgg = 1u << 30, kLookPrefix = 2u << 30, kLookValue = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;  // polls of one predecessor's word before giving up

// SYS: the digit is byte (shift / 8) of the payload's system id instead of
// the key (the extra passes that order several systems).
template <bool SYS>
__device__ __forceinline__ uint32_t sort_digit(uint64_t key, uint32_t val, int shift,
                                               const uint32_t *sys_of) {
  return SYS ? ((sys_of[val] >> shift) & 255u) : (uint32_t)((key >> shift) & 255u);
}

// Digit counts of every pass: hist[p * 256 + d], pass p < 8 the key's byte
// p, passes 8, 9 the bytes of the system id; block counts in shared memory
// (one shared atomic per key and pass), then added to the global counts.
__global__ void __launch_bounds__(kSortThreads) k_sort_hist_all(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ sys_of, int64_t n, int passes, uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[kSortMaxPasses][256];
  for (int k = threadIdx.x; k < kSortMaxPasses * 256; k += kSortThreads) (&h[0][0])[k] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * kSortThreads;
  for (int64_t b = (int64_t)blockIdx.x * kSortThreads; b < n; b += stride) {
    const int64_t i = b + threadIdx.x;
    const bool valid = i < n;
    const uint64_t key = valid ? keys[i] : 0ull;
    const uint32_t sys = (valid && passes > 8) ? sys_of[vals[i]] : 0u;
    for (int p = 0; p < passes; p++) {
      const uint32_t d = !valid ? 256u : p < 8 ? (uint32_t)((key >> (8 * p)) & 255u)
                                               : (sys >> (8 * (p - 8))) & 255u;
      if (valid) atomicAdd(&h[p][d], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < passes * 256; k += kSortThreads) {
    const uint32_t v = (&h[0][0])[k];
    if (v) atomicAdd(&hist[k], v);
  }
}

// Exclusive scan of one value per thread of a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_256(uint32_t v, uint32_t *warp_sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kSortWarps ? warp_sums[lane] : 0u;
    uint32_t winc = w;
#pragma unroll
    for (int o = 1; o < kSortWarps; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    if (lane < kSortWarps) warp_sums[lane] = winc - w;
  }
  __syncthreads();
  return warp_sums[warp] + inc - v;
}

// Publishes the tile's count of digit tid and returns the count of that
// digit in all preceding tiles (decoupled look-back; look[t * 256 + d]).
__device__ __forceinline__ uint32_t sort_look_back(uint32_t *look, uint32_t tile, uint32_t mine,
                                                   int *status) {
  const int tid = threadIdx.x;
  volatile uint32_t *vl = look;
  uint32_t excl = 0;
  if (tile == 0) {
    vl[tid] = kLookPrefix | mine;
    return 0;
  }
  vl[(size_t)tile * 256 + tid] = kLookAgg | mine;
  for (int64_t t = (int64_t)tile - 1; t >= 0; t--) {
    uint32_t w = vl[(size_t)t * 256 + tid];
    for (uint32_t k = 0; (w & ~kLookValue) == 0u; k++) {
      if (k == kSpinLimit) {  // give up: the pass's result is wrong, the call fails
        atomicOr(status, kStSpin);
        w = kLookPrefix;
        break;
      }
      __nanosleep(32);
      w = vl[(size_t)t * 256 + tid];
    }
    excl += w & kLookValue;
    if ((w & ~kLookValue) == kLookPrefix) break;
  }
  vl[(size_t)tile * 256 + tid] = kLookPrefix | ((excl + mine) & kLookValue);
  return excl;
}

// Dynamic shared memory of one pass: the tile's keys, payloads and digits
// in their sorted order (the warps' digit counters alias the key area
// before the keys are placed).
constexpr size_t kSortSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(uint32_t) + 1);
constexpr int kSortPerWarp = kSortTile / kSortWarps;

// One pass: look[t * 256 + d] are the tiles' look-back words and *ctr the
// tile counter, both zero at launch; hist the pass's 256 digit counts.
// Each warp reads a contiguous kSortPerWarp-key run of the tile once into
// registers and ranks it in input order against warp-private digit
// counters (a lane's rank among equal digits of its round from a warp
// match, the round's base from the counter); after the look-back the tile
// is placed in sorted order in shared memory and written out in runs of
// equal digits, consecutive threads to consecutive addresses.
template <bool SYS>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ sys_of, int64_t n, int shift,
    const uint32_t *__restrict__ hist, uint32_t *look, uint32_t *ctr, int *status) {
  extern __shared__ __align__(16) unsigned char sort_smem[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(sort_smem);
  uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kSortTile);
  uint8_t *sdig = reinterpret_cast<uint8_t *>(sval + kSortTile);
  uint32_t *wcnt = reinterpret_cast<uint32_t *>(sort_smem);  // [kSortWarps][256], before placement
  __shared__ uint32_t s_tile;
  __shared__ uint32_t gbase[256], lstart[256];
  __shared__ uint32_t wsum0[kSortWarps], wsum1[kSortWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  if (tid == 0) s_tile = atomicAdd(ctr, 1u);
  for (int k = tid; k < kSortWarps * 256; k += kSortThreads) wcnt[k] = 0u;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t base = (int64_t)tile * kSortTile + (int64_t)warp * kSortPerWarp + lane;
  uint64_t key[kSortRounds];
  uint32_t val[kSortRounds];
  uint32_t dr[kSortRounds];  // digit (256: no key) << 16 | rank
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const int64_t i = base + r * 32;
    const bool valid = i < n;
    key[r] = valid ? kin[i] : 0ull;
    val[r] = valid ? vin[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const bool valid = base + r * 32 < n;
    const uint32_t d = valid ? sort_digit<SYS>(key[r], val[r], shift, sys_of) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0u;
    if (lane == leader && d < 256u) {
      before = wcnt[warp * 256 + d];
      wcnt[warp * 256 + d] = before + (uint32_t)__popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    dr[r] = (d << 16) | (before + (uint32_t)__popc(peers & lt));
    __syncwarp();
  }
  __syncthreads();
  // thread tid: digit tid -- the warps' counts become exclusive offsets
  uint32_t mine = 0u;
#pragma unroll
  for (int w = 0; w < kSortWarps; w++) {
    const uint32_t c = wcnt[w * 256 + tid];
    wcnt[w * 256 + tid] = mine;
    mine += c;
  }
  const uint32_t excl = sort_look_back(look, tile, mine, status);
  gbase[tid] = block_excl_256(hist[tid], wsum0) + excl;
  lstart[tid] = block_excl_256(mine, wsum1);
  __syncthreads();
  // each key's place in the tile's sorted order
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const uint32_t d = dr[r] >> 16;
    if (d < 256u) dr[r] = (d << 16) | (lstart[d] + wcnt[warp * 256 + d] + (dr[r] & 0xffffu));
  }
  __syncthreads();  // the counters' area now takes the keys
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const uint32_t d = dr[r] >> 16;
    if (d < 256u) {
      const uint32_t p = dr[r] & 0xffffu;
      skey[p] = key[r];
      sval[p] = val[r];
      sdig[p] = (uint8_t)d;
    }
  }
  __syncthreads();
  const int64_t rem = n - (int64_t)tile * kSortTile;
  const int cnt = rem < kSortTile ? (int)rem : kSortTile;
  for (int j = tid; j < cnt; j += kSortThreads) {
    const uint32_t d = sdig[j];
    const uint32_t pos = gbase[d] + ((uint32_t)j - lstart[d]);
    kout[pos] = skey[j];
    vout[pos] = sval[j];
  }
}
// ---------------------------------------------------------------------------
// Reorder (Section 4.3 step 3): gather the caller-order FP64 data into Morton
// order, and split positions into FP32 hi/lo pairs (hi = RN(x), lo =
// RN(x - hi)) for the force kernel's group-relative coordinates. The
// conversions run in integer arithmetic (afd_split.cuh), which leaves GB300's
// narrow FP64 unit the three mass products.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split2(double v, float &h, float &l) { afd_split2(v, &h, &l); }

__global__ void __launch_bounds__(kThreads) k_reorder(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ m, int64_t n, const uint32_t *__restrict__ perm,
    double *__restrict__ xs, double *__restrict__ ys, double *__restrict__ zs,
    double *__restrict__ ms, float4 *__restrict__ jhi, float4 *__restrict__ jlo,
    double *__restrict__ mxyz, int *status) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t i = perm[k];
  const double vx = x[i], vy = y[i], vz = z[i], vm = m[i];
  if (!afd_finite_bits(vx) || !afd_finite_bits(vy) || !afd_finite_bits(vz) ||
      !afd_finite_bits(vm))
    atomicOr(status, kStNonFinite);
  xs[k] = vx;
  ys[k] = vy;
  zs[k] = vz;
  ms[k] = vm;
  // the mass moment's products, each rounded as the leaf sum takes them
  mxyz[k] = __dmul_rn(vm, vx);
  mxyz[n + k] = __dmul_rn(vm, vy);
  mxyz[2 * n + k] = __dmul_rn(vm, vz);
  float hx, hy, hz, lx, ly, lz;
  split2(vx, hx, lx);
  split2(vy, hy, ly);
  split2(vz, hz, lz);
  jhi[k] = make_float4(hx, hy, hz, afd_round_f32(vm));
  jlo[k] = make_float4(lx, ly, lz, 0.0f);
}

// ---------------------------------------------------------------------------
// Link (Section 4.3 step 4). The level-l cell holding particle i exists iff
// every ancestor holds more than n_leaf particles (and l <= 21); it is
// started by i iff i is the first particle of its level-l key prefix. With
//   d_i = equal leading digits of keys i-1 and i (-1 for i = 0),
//   c_j = equal leading digits of keys j and j + n_leaf,
//   E_i = min(21, 1 + max_{j in [i-n_leaf, i]} c_j)  (0 when n <= n_leaf),
// particle i starts exactly the cells of levels d_i+1 .. E_i, and E_i is the
// level of its leaf. Emitting cells per particle in (i, level) order gives
// depth-first pre-order directly; cell boundaries come from a binary search
// on the sorted keys, as in the paper.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int common_digits(uint64_t a, uint64_t b) {
  const uint64_t x = a ^ b;
  if (x == 0) return kLevels;
  return (__clzll((long long)x) - 1) / 3;
}

// Range [start, end) of the system holding sorted position i.
__device__ __forceinline__ void sys_range(const uint32_t *sys_s, const int64_t *sys_off,
                                          int64_t n, int64_t i, int64_t &start, int64_t &end) {
  if (sys_s) {
    const uint32_t s = sys_s[i];
    start = sys_off[s];
    end = sys_off[s + 1];
  } else {
    start = 0;
    end = n;
  }
}

// d_i (255 when i starts its system) and c_j (only where j + n_leaf is in
// the same system).
__global__ void __launch_bounds__(kThreads) k_link_dc(const uint64_t *__restrict__ K, int64_t n,
                                                      int n_leaf, const uint32_t *__restrict__ sys_s,
                                                      const int64_t *__restrict__ sys_off,
                                                      uint8_t *__restrict__ dI,
                                                      uint8_t *__restrict__ cJ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t start, end;
  sys_range(sys_s, sys_off, n, i, start, end);
  const uint64_t ki = K[i];
  dI[i] = i == start ? (uint8_t)255 : (uint8_t)common_digits(K[i - 1], ki);
  if (i + n_leaf < end) cJ[i] = (uint8_t)common_digits(ki, K[i + n_leaf]);
}

__global__ void __launch_bounds__(kThreads) k_link_count(const uint8_t *__restrict__ dI,
                                                         const uint8_t *__restrict__ cJ,
                                                         int64_t n, int n_leaf,
                                                         const uint32_t *__restrict__ sys_s,
                                                         const int64_t *__restrict__ sys_off,
                                                         uint8_t *__restrict__ eI,
                                                         uint32_t *__restrict__ cnt,
                                                         unsigned *__restrict__ max_level) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int E = 0;
  if (i < n) {
    int64_t start, end;
    sys_range(sys_s, sys_off, n, i, start, end);
    const int64_t lo = i - n_leaf > start ? i - n_leaf : start;
    const int64_t hi = i < end - n_leaf - 1 ? i : end - n_leaf - 1;
    int mx = -1;
    for (int64_t j = lo; j <= hi; j++) mx = max(mx, (int)cJ[j]);
    E = mx < 0 ? 0 : min(kLevels, mx + 1);
    const int d = dI[i] == 255 ? -1 : (int)dI[i];
    eI[i] = (uint8_t)E;
    cnt[i] = (uint32_t)max(0, E - d);
  }
  // deepest leaf level: one atomic per warp
  const unsigned wm = __reduce_max_sync(0xffffffffu, (unsigned)E);
  if ((threadIdx.x & 31) == 0 && wm > 0) atomicMax(max_level, wm);
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t *K, int64_t lo, int64_t hi,
                                                   uint64_t v) {
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (K[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The same position, found by galloping from lo (first index with K >= v in
// [lo, hi)): cells are mostly small, so the bound is near lo and the probes
// K[lo + 1], K[lo + 3], K[lo + 7], ... stay in a few cache lines before the
// binary search over the last doubling.
__device__ __forceinline__ int64_t gallop_up(const uint64_t *K, int64_t lo, int64_t hi, uint64_t v) {
  int64_t step = 1, prev = lo;
  while (lo < hi && K[lo] < v) {
    prev = lo + 1;
    lo = lo + step < hi ? lo + step : hi;
    step <<= 1;
  }
  return lower_bound_key(K, prev, lo, v);
}

// The first index s in [lo, hi) with K[s] >= v, galloping down from hi - 1
// (a parent cell usually starts a few particles before hi).
__device__ __forceinline__ int64_t gallop_down(const uint64_t *K, int64_t lo, int64_t hi,
                                               uint64_t v) {
  int64_t step = 1, top = hi;
  int64_t q = hi - 1;
  while (q >= lo && K[q] >= v) {
    top = q;
    q = q - step >= lo ? q - step : lo - 1;
    step <<= 1;
  }
  return lower_bound_key(K, q + 1, top, v);
}

// Each particle writes the level and first particle of the cells it starts
// (a few stores, no searches); k_link_cells then completes every cell on a
// thread of its own, so that the long searches of the large cells near the
// root (one particle starts all of them) run side by side.
__global__ void __launch_bounds__(kThreads) k_link_emit(const uint8_t *__restrict__ dI,
                                                        const uint8_t *__restrict__ eI,
                                                        const uint32_t *__restrict__ off,
                                                        int64_t n, uint32_t *__restrict__ level,
                                                        uint32_t *__restrict__ first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d = dI[i] == 255 ? -1 : (int)dI[i];
  const int E = eI[i];
  for (int l = d + 1; l <= E; l++) {
    const uint32_t id = off[i] + (uint32_t)(l - d - 1);
    level[id] = (uint32_t)l;
    first[id] = (uint32_t)i;
  }
}

// Cell id of level l started by particle i: its particle count and skip
// (the end of its key prefix, by a galloping search), its parent (the
// previous cell of the same particle, or the cell of level l - 1 that holds
// i, found by a search back to that prefix's first particle) and its slot
// among the parent's children.
__global__ void __launch_bounds__(kThreads) k_link_cells(
    const uint64_t *__restrict__ K, const uint8_t *__restrict__ dI,
    const uint32_t *__restrict__ off, int64_t n, int64_t n_cells,
    const uint32_t *__restrict__ sys_s, const int64_t *__restrict__ sys_off,
    const uint32_t *__restrict__ level, const uint32_t *__restrict__ first,
    uint32_t *__restrict__ count, uint32_t *__restrict__ skip, uint32_t *__restrict__ parent,
    uint32_t *__restrict__ child) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_cells) return;
  const uint32_t id = (uint32_t)t;
  const int64_t i = first[id];
  if (!AFD_IN(i, n, "link cell first")) return;
  const int l = (int)level[id];
  int64_t sstart, send;
  sys_range(sys_s, sys_off, n, i, sstart, send);
  const int d = dI[i] == 255 ? -1 : (int)dI[i];
  const uint64_t ki = K[i];
  int64_t end = send;
  if (l > 0) {
    const int shift = 3 * (kLevels - l);
    const uint64_t P = ki >> shift;
    end = gallop_up(K, i + 1, send, (P + 1) << shift);
  }
  count[id] = (uint32_t)(end - i);
  skip[id] = off[end];
  uint32_t par = kNone;
  if (l > 0) {
    if (l - 1 >= d + 1) {
      par = id - 1;
    } else {
      const int pshift = 3 * (kLevels - l + 1);
      const uint64_t PP = ki >> pshift;
      const int64_t s = gallop_down(K, sstart, i, PP << pshift);
      const int ds = dI[s] == 255 ? -1 : (int)dI[s];
      par = off[s] + (uint32_t)((l - 1) - ds - 1);
    }
    child[(size_t)par * 8 + ((ki >> (3 * (kLevels - l))) & 7u)] = id;
  }
  parent[id] = par;
}

// ---------------------------------------------------------------------------
// Moments (Section 4.3, bottom-up). One thread per leaf sums its particles
// in Morton order, then climbs: the last child to finish (arrival counter)
// sums the parent's children in octant order. M, S = sum m x, COM = S / M
// (the geometric centre for a massless cell); optional traceless quadrupole
// about the COM with the parallel-axis shift. Finishing a cell also writes
// the superparticle data (COM hi/lo, mass, quadrupole as floats) and the
// walk node (FP32 COM, squared side, first, count, leaf bit).
// ---------------------------------------------------------------------------
struct MomArgs {
  int64_t n_cells;
  const uint32_t *level, *first, *count, *parent, *child;
  const double *xs, *ys, *zs, *ms;
  const double *mxyz;  // m x, m y, m z per particle (3 x n_part)
  const uint64_t *keys;
  const double *root;       // 4 doubles per system
  const uint32_t *sys_s;    // system of each sorted particle (null: one system)
  double *mass, *smom, *com, *quad;
  unsigned *arrive;
  float4 *s_hi, *s_lo, *s_q0, *s_q1, *node_f;
  uint2 *node_i;
  uint4 *block;  // child walk records, 8 per cell (null: not written)
  const uint32_t *leaf_ord;  // leaves by particle count (quadrupole climb only)
  const uint32_t *n_leaves;  // their number (device)
  int quad_on;
  int64_t n_part;  // particles (read only by the self-checking build)
  int *status;     // kStClimb if a climb outruns the tree's depth
};

__device__ __forceinline__ int n_children(const uint32_t *child, uint32_t c) {
  int k = 0;
#pragma unroll
  for (int o = 0; o < 8; o++) k += __ldg(&child[(size_t)c * 8 + o]) != kNone;
  return k;
}

// Leaves ordered by particle count (buckets: counts 1 .. 31, then 32 or
// more), so that the lanes of a warp in the quadrupole climb sum leaves of
// nearly equal length: a leaf's quadrupole is about thirty FP64 operations
// per particle on one lane, and a warp instruction costs GB300's narrow FP64
// unit the same whatever its active lanes (2^22 particles: the tree build
// with quadrupoles 2.97 -> 2.54 ms). The monopole sums keep the cell order:
// there the neighbouring leaves of a warp read neighbouring particles, and
// the count order was not faster. The moments do not depend on the order
// (every cell's sums run in the definition's order on whichever lane takes
// the cell).
constexpr int kLeafBuckets = 32;

__device__ __forceinline__ uint32_t leaf_bucket(uint32_t count) {
  return count >= (uint32_t)kLeafBuckets ? (uint32_t)kLeafBuckets - 1u
                                         : (count > 0u ? count - 1u : 0u);
}

// The order is stable: within a bucket the leaves keep their cell
// (depth-first) order, so a warp's leaves lie close together in space.
// Block b's count of bucket k goes to cnt[k * nb + b]; an exclusive scan of
// cnt (bucket-major) gives every (bucket, block) its first position.
__global__ void __launch_bounds__(kThreads) k_leaf_count(int64_t nc,
                                                         const uint32_t *__restrict__ child,
                                                         const uint32_t *__restrict__ count,
                                                         uint32_t *__restrict__ cnt) {
  __shared__ uint32_t h[kLeafBuckets];
  if (threadIdx.x < kLeafBuckets) h[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && n_children(child, (uint32_t)c) == 0) atomicAdd(&h[leaf_bucket(count[c])], 1u);
  __syncthreads();
  if (threadIdx.x < kLeafBuckets) cnt[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_leaf_place(int64_t nc,
                                                         const uint32_t *__restrict__ child,
                                                         const uint32_t *__restrict__ count,
                                                         const uint32_t *__restrict__ off,
                                                         uint32_t *__restrict__ ord) {
  __shared__ uint32_t wc[kThreads / 32][kLeafBuckets];  // per warp and bucket: leaves, then offsets
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int k = threadIdx.x; k < (kThreads / 32) * kLeafBuckets; k += kThreads) (&wc[0][0])[k] = 0u;
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool leaf = c < nc && n_children(child, (uint32_t)c) == 0;
  const uint32_t b = leaf ? leaf_bucket(count[c]) : (uint32_t)kLeafBuckets;
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  if (leaf && lane == __ffs(peers) - 1) wc[warp][b] = (uint32_t)__popc(peers);
  __syncthreads();
  if (threadIdx.x < kLeafBuckets) {  // exclusive over the warps, then the block's first position
    uint32_t run = off[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) {
      const uint32_t v = wc[w][threadIdx.x];
      wc[w][threadIdx.x] = run;
      run += v;
    }
  }
  __syncthreads();
  if (leaf) ord[wc[warp][b] + (uint32_t)__popc(peers & lt)] = (uint32_t)c;
}

#ifndef AFD_MOM_ACQREL
#define AFD_MOM_ACQREL 1
#endif
// A child's arrival at its parent: one more on the parent's counter; returns
// the count before. With AFD_MOM_ACQREL the addition itself orders memory at
// GPU scope: release for the writes that precede it (the child's sums,
// written by this lane or by lanes of its warp before the warp's barrier),
// acquire for the lane that completes the parent (it, and after the warp's
// barrier the lanes that sum the parent, see every child's sums). Otherwise
// a fence on either side of a relaxed addition does the same.
__device__ __forceinline__ unsigned arrive_at(unsigned *ctr) {
#if AFD_MOM_ACQREL
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
  return old;
#else
  __threadfence();
  const unsigned old = atomicAdd(ctr, 1u);
  __threadfence();
  return old;
#endif
}

__device__ void finish_cell(const MomArgs &a, uint32_t c, double M, const double S[3], bool leaf) {
  const double *root = a.root + (a.sys_s ? 4 * (size_t)a.sys_s[a.first[c]] : 0);
  double g[3];
  if (M != 0.0) {
    for (int d = 0; d < 3; d++) g[d] = __ddiv_rn(S[d], M);
  } else {
    const int l = (int)a.level[c];
    const uint64_t prefix = l > 0 ? a.keys[a.first[c]] >> (3 * (kLevels - l)) : 0ull;
    uint32_t q[3] = {0u, 0u, 0u};
    for (int k = 0; k < l; k++) {
      q[0] |= (uint32_t)((prefix >> (3 * k + 2)) & 1u) << k;
      q[1] |= (uint32_t)((prefix >> (3 * k + 1)) & 1u) << k;
      q[2] |= (uint32_t)((prefix >> (3 * k)) & 1u) << k;
    }
    const double L = root[3];
    const double s = ldexp(L, -l);
    for (int d = 0; d < 3; d++)
      g[d] = __dadd_rn(__dsub_rn(root[d], __dmul_rn(L, 0.5)), __dmul_rn((double)q[d] + 0.5, s));
  }
  a.mass[c] = M;
  for (int d = 0; d < 3; d++) {
    a.smom[(size_t)c * 3 + d] = S[d];
    a.com[(size_t)c * 3 + d] = g[d];
  }
  float h[3], lo[3];
  for (int d = 0; d < 3; d++) split2(g[d], h[d], lo[d]);
  a.s_hi[c] = make_float4(h[0], h[1], h[2], afd_round_f32(M));
  a.s_lo[c] = make_float4(lo[0], lo[1], lo[2], 0.0f);
  const float sd = ldexpf(__double2float_rn(root[3]), -(int)a.level[c]);
  a.node_f[c] = make_float4(h[0], h[1], h[2], __fmul_rn(sd, sd));
  a.node_i[c] = make_uint2(a.first[c], a.count[c] | (leaf ? 0x80000000u : 0u));
}

__device__ void leaf_quad(const MomArgs &a, uint32_t c) {
  const double *g = &a.com[(size_t)c * 3];
  double Q[6] = {0, 0, 0, 0, 0, 0};
  const uint32_t f = a.first[c], e = f + a.count[c];
  for (uint32_t k = f; k < e; k++) {
    const double d0 = __dsub_rn(a.xs[k], g[0]), d1 = __dsub_rn(a.ys[k], g[1]),
                 d2 = __dsub_rn(a.zs[k], g[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    const double mk = a.ms[k];
    Q[0] = __dadd_rn(Q[0], __dmul_rn(mk, __dsub_rn(__dmul_rn(__dmul_rn(3.0, d0), d0), r2)));
    Q[1] = __dadd_rn(Q[1], __dmul_rn(mk, __dsub_rn(__dmul_rn(__dmul_rn(3.0, d1), d1), r2)));
    Q[2] = __dadd_rn(Q[2], __dmul_rn(mk, __dsub_rn(__dmul_rn(__dmul_rn(3.0, d2), d2), r2)));
    Q[3] = __dadd_rn(Q[3], __dmul_rn(mk, __dmul_rn(__dmul_rn(3.0, d0), d1)));
    Q[4] = __dadd_rn(Q[4], __dmul_rn(mk, __dmul_rn(__dmul_rn(3.0, d0), d2)));
    Q[5] = __dadd_rn(Q[5], __dmul_rn(mk, __dmul_rn(__dmul_rn(3.0, d1), d2)));
  }
  for (int q = 0; q < 6; q++) a.quad[(size_t)c * 6 + q] = Q[q];
  a.s_q0[c] = make_float4(__double2float_rn(Q[0]), __double2float_rn(Q[1]),
                          __double2float_rn(Q[2]), __double2float_rn(Q[3]));
  a.s_q1[c] = make_float4(__double2float_rn(Q[4]), __double2float_rn(Q[5]), 0.0f, 0.0f);
}

// Moments in passes. A single climb that finished each cell on the lane of
// its last arriving child would run three correctly rounded FP64 divisions,
// the FP32 splits and the quadrupole sums on a warp with one lane active,
// and GB300's FP64 pipe takes as long for a one-lane warp instruction as for
// a full one. So only the ordered sums M and S climb (k_moments_sums); the
// centres of mass and the FP32 superparticle data follow in one thread per
// cell on full warps (k_moments_finish), the walk's child records in
// another pass (k_moments_blocks, construction steps), and the quadrupoles
// in a second climb (k_moments_quad) that sums six components of a parent
// on six lanes. Each cell's arithmetic is the definition's, in the same
// order.
__global__ void __launch_bounds__(kThreads) k_moments_sums(MomArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t c = (uint32_t)t;
  // climbing: this lane holds a finished cell whose parent it reports to
  bool climbing = t < a.n_cells && n_children(a.child, c) == 0;
  if (climbing) {
    double M = 0.0, S[3] = {0.0, 0.0, 0.0};
    const uint32_t f = a.first[c], e = f + a.count[c];
    if (e > f && !AFD_IN(e - 1, a.n_part, "moments leaf range")) {
      climbing = false;
    } else {
      // the products m x, m y, m z were rounded by the reorder (full warps);
      // here only the ordered sums run on the leaf's lane
      const double *mx = a.mxyz, *my = a.mxyz + a.n_part, *mz = a.mxyz + 2 * a.n_part;
#pragma unroll 4
      for (uint32_t k = f; k < e; k++) {
        M = __dadd_rn(M, a.ms[k]);
        S[0] = __dadd_rn(S[0], mx[k]);
        S[1] = __dadd_rn(S[1], my[k]);
        S[2] = __dadd_rn(S[2], mz[k]);
      }
      a.mass[c] = M;
      for (int d = 0; d < 3; d++) a.smom[(size_t)c * 3 + d] = S[d];
    }
  }
  // The warp climbs together: each lane reports its cell at the parent; the
  // parents this warp completes are summed four lanes each (M, S_x, S_y,
  // S_z: one ordered chain over the octants per lane), eight at a time.
  uint32_t pc = climbing ? a.parent[c] : kNone;  // parent of the climbing cell
  // a cell of level l reaches the root in l climbs: at most kLevels + 1
  // rounds for any tree the link builds (bounded by construction)
  for (int round = 0; __any_sync(0xffffffffu, climbing); round++) {
    if (round > kLevels + 1) {
      if (climbing) atomicOr(a.status, kStClimb);
      break;
    }
    bool won = false;
    if (climbing) {
      const uint32_t p = pc;
      if (p == kNone || !AFD_IN(p, a.n_cells, "moments parent")) {
        climbing = false;
      } else {
        // the child table is read-only here: its loads need not wait for the arrival
        const int nch = n_children(a.child, p);
        const unsigned old = arrive_at(&a.arrive[p]);
        won = (int)old == nch - 1;
        climbing = won;
        if (won) {
          c = p;
          pc = a.parent[p];  // for the next level, in flight while the sums run
        }
      }
    }
    __syncwarp();  // the winners' view of the children reaches the lanes summing them
    unsigned wm = __ballot_sync(0xffffffffu, won);
    while (wm) {
      // the next (up to) eight completed parents: lane 4j + ch takes chain ch
      // of the j-th
      const int j = lane >> 2, ch = lane & 3;
      unsigned rest = wm;
      int src = -1;
      for (int q = 0; q <= j && rest; q++) {
        src = __ffs(rest) - 1;
        rest &= rest - 1;
      }
      const bool mine = src >= 0 && __popc(wm & ((2u << src) - 1u)) == j + 1;
      const uint32_t pj = __shfl_sync(0xffffffffu, c, src < 0 ? 0 : src);
      if (mine) {
        double acc = 0.0;
        for (int o = 0; o < 8; o++) {
          const uint32_t cc = __ldg(&a.child[(size_t)pj * 8 + o]);
          if (cc == kNone || !AFD_IN(cc, a.n_cells, "moments child")) continue;
          acc = __dadd_rn(acc, ch == 0 ? __ldcg(&a.mass[cc])
                                       : __ldcg(&a.smom[(size_t)cc * 3 + (ch - 1)]));
        }
        if (ch == 0) a.mass[pj] = acc;
        else a.smom[(size_t)pj * 3 + (ch - 1)] = acc;
      }
      // drop the parents just summed
      for (int q = 0; q < 8 && wm; q++) wm &= wm - 1;
    }
    __syncwarp();  // the sums are ordered before the climbing lane's fence and arrival
  }
}

// Quadrupoles after the monopole passes (every centre of mass known): leaves
// sum their particles (leaf_quad, one lane per leaf, Morton order), then the
// parents climb with arrival counters like the sums. The completed parents
// of a warp are summed four at a time: a lane per child forms the child's
// six shifted terms Q_c + M_c (3 D_a D_b - r^2 delta_ab) (D = COM_c -
// COM_p), a lane per component adds them in octant order. Every cell's
// arithmetic is the definition's, in the same order, whichever lanes run it.
__global__ void __launch_bounds__(kThreads) k_moments_quad(MomArgs a) {
  // per warp: the shifted terms of the children of four parents
  __shared__ double qstage[kThreads / 32][4][8][6];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool climbing = t < (int64_t)*a.n_leaves;
  uint32_t c = climbing ? a.leaf_ord[t] : 0u;
  if (climbing && !AFD_IN(c, a.n_cells, "quad leaf")) climbing = false;
  if (climbing) {
    const uint32_t f = a.first[c], e = f + a.count[c];
    if (e > f && !AFD_IN(e - 1, a.n_part, "quad leaf range")) climbing = false;
    else leaf_quad(a, c);
  }
  uint32_t pc = climbing ? a.parent[c] : kNone;
  // a cell of level l reaches the root in l climbs: at most kLevels + 1
  // rounds for any tree the link builds (bounded by construction)
  for (int round = 0; __any_sync(0xffffffffu, climbing); round++) {
    if (round > kLevels + 1) {
      if (climbing) atomicOr(a.status, kStClimb);
      break;
    }
    bool won = false;
    if (climbing) {
      const uint32_t p = pc;
      if (p == kNone || !AFD_IN(p, a.n_cells, "quad parent")) {
        climbing = false;
      } else {
        // the child table is read-only here: its loads need not wait for the arrival
        const int nch = n_children(a.child, p);
        const unsigned old = arrive_at(&a.arrive[p]);
        won = (int)old == nch - 1;
        climbing = won;
        if (won) {
          c = p;
          pc = a.parent[p];
        }
      }
    }
    __syncwarp();
    unsigned wm = __ballot_sync(0xffffffffu, won);
    while (wm) {
      // The next (up to) four completed parents: lane 8j + o computes the six
      // shifted terms of child o of the j-th (once per child, not once per
      // component), then lane 8j + q (q < 6) chains component q over the
      // children in octant order, reading the terms from shared memory.
      const int j = lane >> 3, o = lane & 7;
      unsigned rest = wm;
      int src = -1;
      for (int k = 0; k <= j && rest; k++) {
        src = __ffs(rest) - 1;
        rest &= rest - 1;
      }
      const bool mine = src >= 0 && __popc(wm & ((2u << src) - 1u)) == j + 1;
      const uint32_t pj = __shfl_sync(0xffffffffu, c, src < 0 ? 0 : src);
      bool has = false;
      if (mine) {
        const uint32_t cc = __ldg(&a.child[(size_t)pj * 8 + o]);
        if (cc != kNone && AFD_IN(cc, a.n_cells, "quad child")) {
          has = true;
          const double g0 = __ldcg(&a.com[(size_t)pj * 3]), g1 = __ldcg(&a.com[(size_t)pj * 3 + 1]),
                       g2 = __ldcg(&a.com[(size_t)pj * 3 + 2]);
          const double D0 = __dsub_rn(__ldcg(&a.com[(size_t)cc * 3 + 0]), g0);
          const double D1 = __dsub_rn(__ldcg(&a.com[(size_t)cc * 3 + 1]), g1);
          const double D2 = __dsub_rn(__ldcg(&a.com[(size_t)cc * 3 + 2]), g2);
          const double mc = __ldcg(&a.mass[cc]);
          const double r2 =
              __dadd_rn(__dadd_rn(__dmul_rn(D0, D0), __dmul_rn(D1, D1)), __dmul_rn(D2, D2));
          const double D[3] = {D0, D1, D2};
          double *tq = qstage[threadIdx.x >> 5][j][o];
#pragma unroll
          for (int q = 0; q < 6; q++) {
            // the component's two axes (diagonal q < 3: a = b = q)
            const int ax = q < 3 ? q : (q == 5 ? 1 : 0), bx = q < 3 ? q : (q == 3 ? 1 : 2);
            const double p3 = __dmul_rn(__dmul_rn(3.0, D[ax]), D[bx]);
            const double term = q < 3 ? __dsub_rn(p3, r2) : p3;
            tq[q] = __dadd_rn(__ldcg(&a.quad[(size_t)cc * 6 + q]), __dmul_rn(mc, term));
          }
        }
      }
      const unsigned hm = __ballot_sync(0xffffffffu, has);
      __syncwarp();
      if (mine && o < 6) {
        const int q = o;
        double acc = 0.0;
        for (int k = 0; k < 8; k++)
          if ((hm >> (8 * j + k)) & 1u) acc = __dadd_rn(acc, qstage[threadIdx.x >> 5][j][k][q]);
        a.quad[(size_t)pj * 6 + q] = acc;
        float *sq = q < 4 ? reinterpret_cast<float *>(&a.s_q0[pj]) + q
                          : reinterpret_cast<float *>(&a.s_q1[pj]) + (q - 4);
        *sq = __double2float_rn(acc);
        if (q == 4) reinterpret_cast<float *>(&a.s_q1[pj])[2] = 0.0f;
        if (q == 5) reinterpret_cast<float *>(&a.s_q1[pj])[3] = 0.0f;
      }
      __syncwarp();  // the stage is free for the next parents
      for (int k = 0; k < 4 && wm; k++) wm &= wm - 1;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kThreads) k_moments_finish(MomArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_cells) return;
  const uint32_t c = (uint32_t)t;
  const double S[3] = {a.smom[(size_t)c * 3], a.smom[(size_t)c * 3 + 1],
                       a.smom[(size_t)c * 3 + 2]};
  finish_cell(a, c, a.mass[c], S, n_children(a.child, c) == 0);
}

__global__ void __launch_bounds__(kThreads) k_moments_blocks(MomArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_cells) return;
  const uint32_t p = (uint32_t)t;
  if (n_children(a.child, p) == 0) return;
  // the walk's view of p's children: (COM_f32, s^2) and (first, count |
  // leaf, id, mass_f32) per octant slot, id = kNone when empty
  for (int o = 0; o < 8; o++) {
    const uint32_t cc = __ldg(&a.child[(size_t)p * 8 + o]);
    uint4 nf = make_uint4(0u, 0u, 0u, 0u), meta = make_uint4(0u, 0u, kNone, 0u);
    if (cc != kNone && AFD_IN(cc, a.n_cells, "moments block child")) {
      const float4 f = a.node_f[cc];
      const uint2 ni = a.node_i[cc];
      nf = make_uint4(__float_as_uint(f.x), __float_as_uint(f.y), __float_as_uint(f.z),
                      __float_as_uint(f.w));
      meta = make_uint4(ni.x, ni.y, cc, __float_as_uint(a.s_hi[cc].w));  // w: mass (FP32)
    }
    a.block[((size_t)p * 8 + o) * 2] = nf;
    a.block[((size_t)p * 8 + o) * 2 + 1] = meta;
  }
}

// Force-kernel work units of a group of cn particles (see k_unit_fill).
__device__ __forceinline__ uint32_t unit_count(uint32_t cn) { return (cn + 31u) / 32u; }

// ---------------------------------------------------------------------------
// i-groups: the maximal cells holding at most n_grp particles, in
// pre-order; a larger leaf is cut into chunks of n_grp.
// ---------------------------------------------------------------------------
// Group size of the system holding a cell (its first particle).
__device__ __forceinline__ uint32_t group_size(uint32_t n_grp, const uint32_t *sys_grp,
                                               const uint32_t *sys_s, uint32_t first) {
  return sys_grp ? sys_grp[sys_s[first]] : n_grp;
}

__global__ void __launch_bounds__(kThreads) k_group_count(int64_t n_cells,
                                                          const uint32_t *__restrict__ first,
                                                          const uint32_t *__restrict__ count,
                                                          const uint32_t *__restrict__ parent,
                                                          const uint32_t *__restrict__ child,
                                                          uint32_t n_grp_all,
                                                          const uint32_t *__restrict__ sys_grp,
                                                          const uint32_t *__restrict__ sys_s,
                                                          uint32_t *__restrict__ gcnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const uint32_t n_grp = group_size(n_grp_all, sys_grp, sys_s, first[c]);
  const uint32_t cnt = count[c];
  uint32_t g = 0;
  if (cnt <= n_grp) {
    const uint32_t p = parent[c];
    g = (p == kNone || count[p] > n_grp) ? 1u : 0u;
  } else if (n_children(child, (uint32_t)c) == 0) {
    g = (cnt + n_grp - 1) / n_grp;
  }
  gcnt[c] = g;
}

__global__ void __launch_bounds__(kThreads) k_group_fill(
    int64_t n_cells, const uint32_t *__restrict__ first, const uint32_t *__restrict__ count,
    const uint32_t *__restrict__ gcnt, const uint32_t *__restrict__ goff, uint32_t n_grp_all,
    const uint32_t *__restrict__ sys_grp, const uint32_t *__restrict__ sys_s,
    const int64_t *__restrict__ sys_off, const uint32_t *__restrict__ cell_off,
    uint32_t *__restrict__ g_first, uint32_t *__restrict__ g_count,
    uint32_t *__restrict__ g_cell, uint32_t *__restrict__ g_root, uint32_t *__restrict__ u_cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const uint32_t k_n = gcnt[c];
  if (k_n == 0) return;
  const uint32_t n_grp = group_size(n_grp_all, sys_grp, sys_s, first[c]);
  // root cell of the system: the first cell its first particle starts
  const uint32_t root = sys_s ? cell_off[sys_off[sys_s[first[c]]]] : 0u;
  for (uint32_t k = 0; k < k_n; k++) {
    const uint32_t g = goff[c] + k;
    const uint32_t f = first[c] + k * n_grp;
    const uint32_t rem = count[c] - k * n_grp;
    const uint32_t cn = rem < n_grp ? rem : n_grp;
    g_first[g] = f;
    g_count[g] = cn;
    g_cell[g] = (uint32_t)c;
    g_root[g] = root;
    u_cnt[g] = unit_count(cn);
  }
}

// Force-kernel work units of a group: one per 32 particles; the last one,
// holding r < 32 particles, splits its warp into S = 4 (r <= 8) or S = 2
// (r <= 16) j-streams. info = (group, first offset | log2(S) << 16).
__global__ void __launch_bounds__(kThreads) k_unit_fill(int64_t n_groups,
                                                        const uint32_t *__restrict__ g_count,
                                                        const uint32_t *__restrict__ u_off,
                                                        uint2 *__restrict__ u_info) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const uint32_t cn = g_count[g];
  uint32_t k = 0;
  for (uint32_t u = u_off[g]; u < u_off[g + 1]; u++, k++) {
    const uint32_t r = cn - 32u * k;
    uint32_t sidx = r >= 32u ? 0u : (r <= 8u ? 2u : (r <= 16u ? 1u : 0u));
    if (sidx > AFD_MAX_SIDX) sidx = AFD_MAX_SIDX;
    u_info[u] = make_uint2((uint32_t)g, (32u * k) | (sidx << 16));
  }
}

// Tight FP64 box per group (one warp per group; min/max are exact) and its
// FP32 copy for the opening criterion.
__global__ void __launch_bounds__(kThreads) k_group_box(
    int64_t n_groups, const uint32_t *__restrict__ g_first, const uint32_t *__restrict__ g_count,
    const double *__restrict__ xs, const double *__restrict__ ys, const double *__restrict__ zs,
    double *__restrict__ box, float *__restrict__ boxf) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_groups) return;
  const uint32_t f = g_first[g], e = f + g_count[g];
  unsigned long long klo[3] = {~0ull, ~0ull, ~0ull}, khi[3] = {0ull, 0ull, 0ull};
  for (uint32_t k = f + lane; k < e; k += 32) {
    const double v[3] = {xs[k], ys[k], zs[k]};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const unsigned long long q = okey(v[d]);
      klo[d] = min(klo[d], q);
      khi[d] = max(khi[d], q);
    }
  }
  double lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    lo[d] = okey_value(warp_min_key(klo[d]));
    hi[d] = okey_value(warp_max_key(khi[d]));
  }
  if (lane != 0) return;
  for (int d = 0; d < 3; d++) {
    box[g * 6 + d] = lo[d];
    box[g * 6 + 3 + d] = hi[d];
    boxf[g * 6 + d] = __double2float_rn(lo[d]);
    boxf[g * 6 + 3 + d] = __double2float_rn(hi[d]);
  }
}

inline int ck() { return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA; }

}  // namespace

#define AFD_TRY(x)            \
  do {                        \
    int _s = (x);             \
    if (_s != AFD_OK) return _s; \
  } while (0)

int launch_root(afd_ctx *c, const double *x, const double *y, const double *z, const double *m,
                int64_t n) {
  AFD_TRY(reserve(c->root, sizeof(double) * 4 * (size_t)c->n_sys));
  AFD_TRY(reserve(c->red_part, sizeof(double) * 6 * kRootBlocks));
  if (c->n_sys > 1) {
    // tiles of at most kRootTile particles that never cross a system
    std::vector<int4> tiles;
    std::vector<int> first(c->n_sys + 1, 0);
    for (int sy = 0; sy < c->n_sys; sy++) {
      first[sy] = (int)tiles.size();
      for (int64_t b = c->sys_off_h[sy]; b < c->sys_off_h[sy + 1]; b += kRootTile) {
        const int64_t e = b + kRootTile < c->sys_off_h[sy + 1] ? b + kRootTile : c->sys_off_h[sy + 1];
        tiles.push_back(make_int4(sy, (int)b, (int)e, 0));
      }
    }
    first[c->n_sys] = (int)tiles.size();
    const size_t tb = sizeof(int4) * tiles.size(), fb = sizeof(int) * first.size();
    AFD_TRY(reserve(c->root_tiles, tb + fb + 16));
    AFD_TRY(reserve(c->red_part, sizeof(double) * 6 * (tiles.size() + 1)));
    AFD_TRY(reserve(c->sys_of, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)));
    char *tp = static_cast<char *>(c->root_tiles.p);
    if ((tb && cudaMemcpyAsync(tp, tiles.data(), tb, cudaMemcpyHostToDevice, c->stream) !=
                   cudaSuccess) ||
        cudaMemcpyAsync(tp + tb, first.data(), fb, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
      return AFD_ERR_CUDA;
    if (!tiles.empty()) {
      k_root_tiles<<<(unsigned)tiles.size(), kThreads, 0, c->stream>>>(
          x, y, z, m, reinterpret_cast<const int4 *>(tp), ptr<unsigned long long>(c->red_part),
          ptr<int>(c->status));
      c->launches++;
    }
    k_root_final<<<(unsigned)c->n_sys, kThreads, 0, c->stream>>>(
        ptr<unsigned long long>(c->red_part), reinterpret_cast<const int *>(tp + tb),
        ptr<double>(c->root), ptr<int>(c->status));
    c->launches++;
    if (n > 0) {
      k_sys_of<<<blocks_for(n), kThreads, 0, c->stream>>>(ptr<int64_t>(c->sys_off_d), c->n_sys, n,
                                                          ptr<uint32_t>(c->sys_of));
      c->launches++;
    }
    return ck();
  }
  if (n == 0) {
    const double r[4] = {0.0, 0.0, 0.0, 1.0};
    return cudaMemcpyAsync(c->root.p, r, sizeof(r), cudaMemcpyHostToDevice, c->stream) == cudaSuccess
               ? AFD_OK
               : AFD_ERR_CUDA;
  }
  int64_t nb = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (nb > kRootBlocks) nb = kRootBlocks;
  k_root<<<(unsigned)nb, kThreads, 0, c->stream>>>(x, y, z, m, n,
                                                  ptr<unsigned long long>(c->red_part),
                                                  ptr<unsigned>(c->red_count),
                                                  ptr<double>(c->root), ptr<int>(c->status));
  c->launches++;
  return ck();
}

int launch_keys(afd_ctx *c, const double *x, const double *y, const double *z, int64_t n) {
  AFD_TRY(reserve(c->keys, sizeof(uint64_t) * n));
  AFD_TRY(reserve(c->perm, sizeof(uint32_t) * n));
  if (n == 0) return AFD_OK;
  k_keys<<<blocks_for(n), kThreads, 0, c->stream>>>(
      x, y, z, n, ptr<double>(c->root), c->n_sys > 1 ? ptr<uint32_t>(c->sys_of) : nullptr,
      ptr<uint64_t>(c->keys), ptr<uint32_t>(c->perm));
  c->launches++;
  return ck();
}

int launch_sort(afd_ctx *c, int64_t n) {
  if (c->n_sys > 1) AFD_TRY(reserve(c->sys_s, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)));
  if (n <= 1) {
    if (c->n_sys > 1 && n == 1) {
      k_sys_of<<<1, kThreads, 0, c->stream>>>(ptr<int64_t>(c->sys_off_d), c->n_sys, n,
                                             ptr<uint32_t>(c->sys_s));
      c->launches++;
    }
    return ck();
  }
  const int num_tiles = (int)((n + kSortTile - 1) / kSortTile);
  // eight passes over the key, then (several systems) one or two passes over
  // the system id: stable, so the result is ordered by (system, key)
  const int sys_passes = c->n_sys > 256 ? 2 : (c->n_sys > 1 ? 1 : 0);
  const int passes = 8 + sys_passes;
  // look-back words of one pass (256 per tile) and its tile counter; all
  // passes' at once when that stays small, else one pass's, cleared per pass
  const size_t look_words = (size_t)256 * num_tiles + 64;
  const bool per_pass = (size_t)passes * look_words * sizeof(uint32_t) > ((size_t)32 << 20);
  const int slices = per_pass ? 1 : passes;
  AFD_TRY(reserve(c->keys2, sizeof(uint64_t) * n));
  AFD_TRY(reserve(c->perm2, sizeof(uint32_t) * n));
  AFD_TRY(reserve(c->sort_cnt, sizeof(uint32_t) * 256 * kSortMaxPasses));
  AFD_TRY(reserve(c->sort_off, sizeof(uint32_t) * look_words * slices));
  uint64_t *ka = ptr<uint64_t>(c->keys), *kb = ptr<uint64_t>(c->keys2);
  uint32_t *va = ptr<uint32_t>(c->perm), *vb = ptr<uint32_t>(c->perm2);
  const uint32_t *sys_of = c->n_sys > 1 ? ptr<uint32_t>(c->sys_of) : nullptr;
  uint32_t *hist = ptr<uint32_t>(c->sort_cnt), *look = ptr<uint32_t>(c->sort_off);
  if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256 * passes, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  if (!per_pass &&
      cudaMemsetAsync(look, 0, sizeof(uint32_t) * look_words * slices, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  const size_t sort_smem = kSortSmem;
  {
    static bool attr_set[8] = {false, false, false, false, false, false, false, false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 8 || !attr_set[dev]) {
      if (cudaFuncSetAttribute(k_sort_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortSmem) != cudaSuccess ||
          cudaFuncSetAttribute(k_sort_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortSmem) != cudaSuccess)
        return AFD_ERR_CUDA;
      if (dev >= 0 && dev < 8) attr_set[dev] = true;
    }
  }
  {
    const int64_t want = (n + kSortThreads - 1) / kSortThreads;
    const unsigned nb = (unsigned)(want < 152 * 4 ? want : 152 * 4);
    k_sort_hist_all<<<nb, kSortThreads, 0, c->stream>>>(ka, va, sys_of, n, passes, hist);
    c->launches++;
    AFD_TRY(ck());
  }
  for (int pass = 0; pass < passes; pass++) {
    const bool sys = pass >= 8;
    const int shift = sys ? 8 * (pass - 8) : 8 * pass;
    uint32_t *lk = look + (per_pass ? 0 : (size_t)pass * look_words);
    if (per_pass &&
        cudaMemsetAsync(lk, 0, sizeof(uint32_t) * look_words, c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    uint32_t *ctr = lk + (size_t)256 * num_tiles;
    if (sys)
      k_sort_pass<true><<<num_tiles, kSortThreads, sort_smem, c->stream>>>(
          ka, va, kb, vb, sys_of, n, shift, hist + 256 * pass, lk, ctr, ptr<int>(c->status));
    else
      k_sort_pass<false><<<num_tiles, kSortThreads, sort_smem, c->stream>>>(
          ka, va, kb, vb, sys_of, n, shift, hist + 256 * pass, lk, ctr, ptr<int>(c->status));
    c->launches++;
    AFD_TRY(ck());
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  if ((8 + sys_passes) & 1) {  // the result sits in the ping-pong buffers
    std::swap(c->keys, c->keys2);
    std::swap(c->perm, c->perm2);
  }
  if (c->n_sys > 1) {
    // sorted positions keep each system's range
    k_sys_of<<<blocks_for(n), kThreads, 0, c->stream>>>(ptr<int64_t>(c->sys_off_d), c->n_sys, n,
                                                        ptr<uint32_t>(c->sys_s));
    c->launches++;
  }
  return ck();
}

int launch_reorder(afd_ctx *c, const double *x, const double *y, const double *z,
                   const double *m, int64_t n) {
  for (afd::DevBuf *b : {&c->xs, &c->ys, &c->zs, &c->ms}) AFD_TRY(reserve(*b, sizeof(double) * n));
  AFD_TRY(reserve(c->jhi, sizeof(float4) * n));
  AFD_TRY(reserve(c->jlo, sizeof(float4) * n));
  AFD_TRY(reserve(c->mxyz, sizeof(double) * 3 * n));
  if (n == 0) return AFD_OK;
  k_reorder<<<blocks_for(n), kThreads, 0, c->stream>>>(
      x, y, z, m, n, ptr<uint32_t>(c->perm), ptr<double>(c->xs), ptr<double>(c->ys),
      ptr<double>(c->zs), ptr<double>(c->ms), ptr<float4>(c->jhi), ptr<float4>(c->jlo),
      ptr<double>(c->mxyz), ptr<int>(c->status));
  c->launches++;
  return ck();
}

int launch_link(afd_ctx *c, int64_t n) {
  AFD_TRY(reserve(c->lk_d, n));
  AFD_TRY(reserve(c->lk_c, n));
  AFD_TRY(reserve(c->lk_e, n));
  AFD_TRY(reserve(c->lk_cnt, sizeof(uint32_t) * n));
  AFD_TRY(reserve(c->lk_off, sizeof(uint32_t) * (n + 1)));
  AFD_TRY(reserve(c->u64acc, sizeof(uint64_t) * 4));
  if (n == 0) {
    c->n_cells = 0;
    c->max_level = 0;
    return AFD_OK;
  }
  const int n_leaf = c->cfg.n_leaf;
  unsigned *maxl = ptr<unsigned>(c->u64acc);
  if (cudaMemsetAsync(maxl, 0, sizeof(unsigned), c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  const uint32_t *sys_s = c->n_sys > 1 ? ptr<uint32_t>(c->sys_s) : nullptr;
  const int64_t *sys_off = ptr<int64_t>(c->sys_off_d);
  k_link_dc<<<blocks_for(n), kThreads, 0, c->stream>>>(ptr<uint64_t>(c->keys), n, n_leaf, sys_s,
                                                       sys_off, ptr<uint8_t>(c->lk_d),
                                                       ptr<uint8_t>(c->lk_c));
  c->launches++;
  k_link_count<<<blocks_for(n), kThreads, 0, c->stream>>>(
      ptr<uint8_t>(c->lk_d), ptr<uint8_t>(c->lk_c), n, n_leaf, sys_s, sys_off,
      ptr<uint8_t>(c->lk_e), ptr<uint32_t>(c->lk_cnt), maxl);
  c->launches++;
  AFD_TRY(ck());
  AFD_TRY(scan_u32(c, ptr<uint32_t>(c->lk_cnt), ptr<uint32_t>(c->lk_off), n));
  uint32_t *pin = static_cast<uint32_t *>(c->pinned);
  cudaMemcpyAsync(pin, ptr<uint32_t>(c->lk_off) + n, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                  c->stream);
  cudaMemcpyAsync(pin + 1, maxl, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  const int64_t nc = pin[0];
  c->n_cells = nc;
  c->max_level = (int)pin[1];
  const size_t u = sizeof(uint32_t) * (size_t)nc;
  for (afd::DevBuf *b : {&c->c_level, &c->c_first, &c->c_count, &c->c_skip, &c->c_parent,
                         &c->c_arrive})
    AFD_TRY(reserve(*b, u));
  AFD_TRY(reserve(c->c_child, u * 8));
  if (cudaMemsetAsync(c->c_child.p, 0xff, u * 8, c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  k_link_emit<<<blocks_for(n), kThreads, 0, c->stream>>>(
      ptr<uint8_t>(c->lk_d), ptr<uint8_t>(c->lk_e), ptr<uint32_t>(c->lk_off), n,
      ptr<uint32_t>(c->c_level), ptr<uint32_t>(c->c_first));
  k_link_cells<<<blocks_for(nc), kThreads, 0, c->stream>>>(
      ptr<uint64_t>(c->keys), ptr<uint8_t>(c->lk_d), ptr<uint32_t>(c->lk_off), n, nc, sys_s,
      sys_off, ptr<uint32_t>(c->c_level), ptr<uint32_t>(c->c_first), ptr<uint32_t>(c->c_count),
      ptr<uint32_t>(c->c_skip), ptr<uint32_t>(c->c_parent), ptr<uint32_t>(c->c_child));
  c->launches += 2;
  c->leaf_ord_ok = false;  // a new topology: the leaf order is made when first needed
  return ck();
}

int launch_moments(afd_ctx *c, bool child_blocks, bool need_q) {
  const int64_t nc = c->n_cells;
  if (child_blocks) AFD_TRY(reserve(c->c_block, sizeof(uint4) * 16 * (size_t)nc));
  AFD_TRY(reserve(c->c_mass, sizeof(double) * nc));
  AFD_TRY(reserve(c->c_smom, sizeof(double) * 3 * nc));
  AFD_TRY(reserve(c->c_com, sizeof(double) * 3 * nc));
  AFD_TRY(reserve(c->c_quad, sizeof(double) * 6 * nc));
  for (afd::DevBuf *b : {&c->s_hi, &c->s_lo, &c->s_q0, &c->s_q1, &c->node_f})
    AFD_TRY(reserve(*b, sizeof(float4) * nc));
  AFD_TRY(reserve(c->node_i, sizeof(uint2) * nc));
  if (nc == 0) return AFD_OK;
  if (cudaMemsetAsync(c->c_arrive.p, 0, sizeof(unsigned) * nc, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  // quadrupoles for the far field, and (construction steps) for the learned
  // opening criterion; without either they are zero in the exports
  const bool quad_on = c->cfg.multipole || need_q;
  c->moments_current = true;
  c->q_current = quad_on;
  c->blocks_current = child_blocks;
  if (!quad_on && !c->cfg.mac) {
    if (cudaMemsetAsync(c->c_quad.p, 0, sizeof(double) * 6 * nc, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->s_q0.p, 0, sizeof(float4) * nc, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->s_q1.p, 0, sizeof(float4) * nc, c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
  }
  MomArgs a;
  a.n_cells = nc;
  a.level = ptr<uint32_t>(c->c_level);
  a.first = ptr<uint32_t>(c->c_first);
  a.count = ptr<uint32_t>(c->c_count);
  a.parent = ptr<uint32_t>(c->c_parent);
  a.child = ptr<uint32_t>(c->c_child);
  a.xs = ptr<double>(c->xs);
  a.ys = ptr<double>(c->ys);
  a.zs = ptr<double>(c->zs);
  a.ms = ptr<double>(c->ms);
  a.mxyz = ptr<double>(c->mxyz);
  a.keys = ptr<uint64_t>(c->keys);
  a.root = ptr<double>(c->root);
  a.sys_s = c->n_sys > 1 ? ptr<uint32_t>(c->sys_s) : nullptr;
  a.mass = ptr<double>(c->c_mass);
  a.smom = ptr<double>(c->c_smom);
  a.com = ptr<double>(c->c_com);
  a.quad = ptr<double>(c->c_quad);
  a.arrive = ptr<unsigned>(c->c_arrive);
  a.s_hi = ptr<float4>(c->s_hi);
  a.s_lo = ptr<float4>(c->s_lo);
  a.s_q0 = ptr<float4>(c->s_q0);
  a.s_q1 = ptr<float4>(c->s_q1);
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.block = child_blocks ? ptr<uint4>(c->c_block) : nullptr;
  const bool leaf_order = quad_on;
  const unsigned nbl = blocks_for(nc);
  if (leaf_order && !c->leaf_ord_ok) {  // the leaves by particle count (stable), for the quadrupoles
    const size_t m = (size_t)kLeafBuckets * nbl;
    AFD_TRY(reserve(c->leaf_ord, sizeof(uint32_t) * (size_t)nc));
    AFD_TRY(reserve(c->leaf_aux, sizeof(uint32_t) * (2 * m + 1)));
    uint32_t *cnt = ptr<uint32_t>(c->leaf_aux), *off = cnt + m;
    k_leaf_count<<<nbl, kThreads, 0, c->stream>>>(nc, ptr<uint32_t>(c->c_child),
                                                   ptr<uint32_t>(c->c_count), cnt);
    c->launches++;
    AFD_TRY(ck());
    AFD_TRY(scan_u32(c, cnt, off, (int64_t)m));
    k_leaf_place<<<nbl, kThreads, 0, c->stream>>>(nc, ptr<uint32_t>(c->c_child),
                                                   ptr<uint32_t>(c->c_count), off,
                                                   ptr<uint32_t>(c->leaf_ord));
    c->launches++;
    AFD_TRY(ck());
    c->leaf_ord_ok = true;
  }
  a.leaf_ord = leaf_order ? ptr<uint32_t>(c->leaf_ord) : nullptr;
  a.n_leaves = leaf_order ? ptr<uint32_t>(c->leaf_aux) + 2 * (size_t)kLeafBuckets * nbl : nullptr;
  a.quad_on = quad_on;
  a.n_part = c->n;
  a.status = ptr<int>(c->status);
  k_moments_sums<<<blocks_for(nc), kThreads, 0, c->stream>>>(a);
  k_moments_finish<<<blocks_for(nc), kThreads, 0, c->stream>>>(a);
  c->launches += 2;
  if (a.block) {
    k_moments_blocks<<<blocks_for(nc), kThreads, 0, c->stream>>>(a);
    c->launches++;
  }
  if (quad_on) {
    if (cudaMemsetAsync(c->c_arrive.p, 0, sizeof(unsigned) * nc, c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    k_moments_quad<<<blocks_for(nc), kThreads, 0, c->stream>>>(a);
    c->launches++;
  }
  return ck();
}

int launch_groups(afd_ctx *c) {
  const int64_t nc = c->n_cells;
  AFD_TRY(reserve(c->g_cnt, sizeof(uint32_t) * nc));
  AFD_TRY(reserve(c->g_off, sizeof(uint32_t) * (nc + 1)));
  if (nc == 0) {
    c->n_groups = 0;
    c->n_units = 0;
    return AFD_OK;
  }
  const uint32_t n_grp = (uint32_t)c->cfg.n_grp;
  const uint32_t *sys_s = c->n_sys > 1 ? ptr<uint32_t>(c->sys_s) : nullptr;
  const uint32_t *sys_grp = (c->n_sys > 1 && !c->sys_grp_h.empty()) ? ptr<uint32_t>(c->sys_grp_d)
                                                                     : nullptr;
  k_group_count<<<blocks_for(nc), kThreads, 0, c->stream>>>(
      nc, ptr<uint32_t>(c->c_first), ptr<uint32_t>(c->c_count), ptr<uint32_t>(c->c_parent),
      ptr<uint32_t>(c->c_child), n_grp, sys_grp, sys_s, ptr<uint32_t>(c->g_cnt));
  c->launches++;
  AFD_TRY(ck());
  AFD_TRY(scan_u32(c, ptr<uint32_t>(c->g_cnt), ptr<uint32_t>(c->g_off), nc));
  uint32_t *pin = static_cast<uint32_t *>(c->pinned);
  cudaMemcpyAsync(pin, ptr<uint32_t>(c->g_off) + nc, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                  c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  const int64_t ng = pin[0];
  c->n_groups = ng;
  for (afd::DevBuf *b : {&c->g_first, &c->g_count, &c->g_cell, &c->g_root, &c->g_self, &c->u_cnt})
    AFD_TRY(reserve(*b, sizeof(uint32_t) * ng));
  AFD_TRY(reserve(c->u_off, sizeof(uint32_t) * (ng + 1)));
  AFD_TRY(reserve(c->g_box, sizeof(double) * 6 * ng));
  AFD_TRY(reserve(c->g_boxf, sizeof(float) * 6 * ng));
  k_group_fill<<<blocks_for(nc), kThreads, 0, c->stream>>>(
      nc, ptr<uint32_t>(c->c_first), ptr<uint32_t>(c->c_count), ptr<uint32_t>(c->g_cnt),
      ptr<uint32_t>(c->g_off), n_grp, sys_grp, sys_s, ptr<int64_t>(c->sys_off_d),
      ptr<uint32_t>(c->lk_off), ptr<uint32_t>(c->g_first), ptr<uint32_t>(c->g_count),
      ptr<uint32_t>(c->g_cell), ptr<uint32_t>(c->g_root), ptr<uint32_t>(c->u_cnt));
  c->launches++;
  AFD_TRY(ck());
  AFD_TRY(scan_u32(c, ptr<uint32_t>(c->u_cnt), ptr<uint32_t>(c->u_off), ng));
  cudaMemcpyAsync(pin, ptr<uint32_t>(c->u_off) + ng, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                  c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  c->n_units = pin[0];
  AFD_TRY(reserve(c->u_info, sizeof(uint2) * c->n_units));
  k_unit_fill<<<blocks_for(ng), kThreads, 0, c->stream>>>(ng, ptr<uint32_t>(c->g_count),
                                                          ptr<uint32_t>(c->u_off),
                                                          ptr<uint2>(c->u_info));
  c->launches++;
  return ck();
}

int launch_group_boxes(afd_ctx *c) {
  const int64_t ng = c->n_groups;
  if (ng == 0) return AFD_OK;
  k_group_box<<<blocks_for(ng * 32), kThreads, 0, c->stream>>>(
      ng, ptr<uint32_t>(c->g_first), ptr<uint32_t>(c->g_count), ptr<double>(c->xs),
      ptr<double>(c->ys), ptr<double>(c->zs), ptr<double>(c->g_box), ptr<float>(c->g_boxf));
  c->launches++;
  return ck();
}

}  // namespace afd
