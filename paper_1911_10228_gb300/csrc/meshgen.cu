// On-device refinement of one mesh level (Sec. 3.1, Eq. ref_crit): a block of
// level l is refined where its source exceeds alpha^(L_R - l) times the
// largest |source| on the level.  The refined blocks' children form the next
// level, and the closure of the mesh needs every refined block's 26 same-level
// neighbours (Sec. 3: the buffer around a refined region), so the neighbours
// missing from the level are listed too.  Outputs are in Morton order.
//
// Morton order: blocks compare by the key that interleaves the bits of
// (x + 2^20, y + 2^20, z + 2^20), bit i of x at key bit 3i + 2, of y at 3i + 1,
// of z at 3i (|coordinates| < 2^20, 21 bits per axis).  Keys are sorted by a
// stable least-significant-bit-first split per bit, run only for the bits that
// vary among the keys (their OR differs from their AND).
#include <cstdint>
#include <utility>
#include <vector>

#include "flgf.h"
#include "internal.h"

namespace flgf {

namespace {

constexpr int kMgThreads = 1024;         // scan tile
constexpr int kMgCoordBias = 1 << 20;    // coordinates + bias are in [0, 2^21)
constexpr int kMgMaxKeys = 1 << 24;      // one-CTA scan of tile sums: <= 16384 tiles

__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x1f00000000ffffull;
  x = (x | (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}
__host__ __device__ inline uint64_t morton_key(int x, int y, int z) {
  return (spread3((uint32_t)(x + kMgCoordBias)) << 2) | (spread3((uint32_t)(y + kMgCoordBias)) << 1) |
         spread3((uint32_t)(z + kMgCoordBias));
}
__device__ inline void morton_decode(uint64_t k, int32_t* c) {
  c[0] = (int32_t)compact3(k >> 2) - kMgCoordBias;
  c[1] = (int32_t)compact3(k >> 1) - kMgCoordBias;
  c[2] = (int32_t)compact3(k) - kMgCoordBias;
}

// max |f| over each block (one CTA per block)
template <typename R>
__global__ void block_absmax_kernel(const R* __restrict__ f, int n3, R* __restrict__ bmax) {
  __shared__ R red[256];
  const R* b = f + (size_t)blockIdx.x * n3;
  R m = R(0);
  for (int i = threadIdx.x; i < n3; i += blockDim.x) m = fmax(m, fabs(b[i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) bmax[blockIdx.x] = red[0];
}

// one CTA: the level maximum, then the flags (comparison in FP64)
template <typename R>
__global__ void flag_kernel(const R* __restrict__ bmax, int n, double rel, uint8_t* __restrict__ flags,
                            uint32_t* __restrict__ nflag) {
  __shared__ double red[kMgThreads];
  __shared__ uint32_t cnt;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, (double)bmax[i]);
  red[threadIdx.x] = m;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double thr = rel * red[0];
  const bool any = red[0] > 0.0;
  uint32_t local = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint8_t v = any && (double)bmax[i] > thr;
    flags[i] = v;
    local += v;
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  if (threadIdx.x == 0) *nflag = cnt;
}

// candidates of the flagged blocks: 8 children keys or 26 neighbour keys each
// (written at slot rank * per + j; rank = exclusive prefix of the flags)
__global__ void emit_kernel(const int32_t* __restrict__ coords, const uint8_t* __restrict__ flags,
                            const uint32_t* __restrict__ rank, int n, int children, uint64_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flags[i]) return;
  const int x = coords[3 * i], y = coords[3 * i + 1], z = coords[3 * i + 2];
  if (children) {
    for (int a = 0; a < 8; ++a)
      out[(size_t)rank[i] * 8 + a] = morton_key(2 * x + (a >> 2), 2 * y + ((a >> 1) & 1), 2 * z + (a & 1));
  } else {
    int j = 0;
    for (int e = 0; e < 27; ++e) {
      if (e == 13) continue;
      out[(size_t)rank[i] * 26 + j++] = morton_key(x + e / 9 - 1, y + (e / 3) % 3 - 1, z + e % 3 - 1);
    }
  }
}

// 1 in *bad when a coordinate is outside (-2^19, 2^19) (children must fit the keys)
__global__ void check_coords_kernel(const int32_t* __restrict__ coords, int n, uint32_t* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const int v = coords[i];
  if (v <= -(kMgCoordBias >> 1) || v >= (kMgCoordBias >> 1)) atomicOr(bad, 1u);
}

__global__ void level_keys_kernel(const int32_t* __restrict__ coords, int n, uint64_t* __restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = morton_key(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
}

// OR and AND of all keys (one CTA): the bits that vary
__global__ void key_bits_kernel(const uint64_t* __restrict__ keys, int n, uint64_t* __restrict__ out) {
  __shared__ unsigned long long o, a;
  if (threadIdx.x == 0) { o = 0ull; a = ~0ull; }
  __syncthreads();
  unsigned long long lo = 0ull, la = ~0ull;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { lo |= keys[i]; la &= keys[i]; }
  atomicOr(&o, lo);
  atomicAnd(&a, la);
  __syncthreads();
  if (threadIdx.x == 0) { out[0] = o; out[1] = a; }
}

// keep[i] for a predicate; rank by exclusive scan
// (a) per-tile scan of 0/1 values, tile sums
__global__ void scan_tiles_kernel(const uint8_t* __restrict__ keep, int n, uint32_t* __restrict__ rank,
                                  uint32_t* __restrict__ tile_sum) {
  __shared__ uint32_t s[kMgThreads];
  const int i = blockIdx.x * kMgThreads + threadIdx.x;
  const uint32_t v = i < n ? keep[i] : 0u;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = 1; w < kMgThreads; w <<= 1) {  // Hillis-Steele inclusive scan
    const uint32_t t = threadIdx.x >= (unsigned)w ? s[threadIdx.x - w] : 0u;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) rank[i] = s[threadIdx.x] - v;
  if (threadIdx.x == kMgThreads - 1) tile_sum[blockIdx.x] = s[threadIdx.x];
}
// (b) one CTA: exclusive scan of the tile sums in place, total at [ntiles]
__global__ void scan_sums_kernel(uint32_t* __restrict__ tile_sum, int ntiles) {
  __shared__ uint32_t s[kMgThreads];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += kMgThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < ntiles ? tile_sum[i] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = 1; w < kMgThreads; w <<= 1) {
      const uint32_t t = threadIdx.x >= (unsigned)w ? s[threadIdx.x - w] : 0u;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < ntiles) tile_sum[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kMgThreads - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}
// (c) rank += tile offset
__global__ void scan_add_kernel(uint32_t* __restrict__ rank, int n, const uint32_t* __restrict__ tile_off) {
  const int i = blockIdx.x * kMgThreads + threadIdx.x;
  if (i < n) rank[i] += tile_off[blockIdx.x];
}

// stable split on one bit: zeros first (in order), then ones
__global__ void bit_kernel(const uint64_t* __restrict__ keys, int n, int bit, uint8_t* __restrict__ zero) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) zero[i] = !((keys[i] >> bit) & 1ull);
}
__global__ void split_scatter_kernel(const uint64_t* __restrict__ in, int n, const uint8_t* __restrict__ zero,
                                     const uint32_t* __restrict__ rank, const uint32_t* __restrict__ nzero,
                                     uint64_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t z = *nzero;
  out[zero[i] ? rank[i] : z + ((uint32_t)i - rank[i])] = in[i];
}

// keep[i]: first of its run of equal sorted keys, and (when lvl != null) not a
// key of the sorted level list
__global__ void select_kernel(const uint64_t* __restrict__ keys, int n, const uint64_t* __restrict__ lvl, int nl,
                              uint8_t* __restrict__ keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  bool v = i == 0 || keys[i - 1] != k;
  if (v && lvl) {
    int lo = 0, hi = nl;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (lvl[mid] < k) lo = mid + 1; else hi = mid;
    }
    v = !(lo < nl && lvl[lo] == k);
  }
  keep[i] = v;
}
__global__ void compact_decode_kernel(const uint64_t* __restrict__ keys, int n, const uint8_t* __restrict__ keep,
                                      const uint32_t* __restrict__ rank, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && keep[i]) morton_decode(keys[i], out + 3 * (size_t)rank[i]);
}

// scratch for lists of up to n keys
struct MgWork {
  uint64_t *k0 = nullptr, *k1 = nullptr, *lvl = nullptr, *bits = nullptr;
  uint8_t* f8 = nullptr;
  uint32_t *rank = nullptr, *tiles = nullptr, *cnt = nullptr;
};

inline int nblk_of(size_t n, int t) { return (int)((n + t - 1) / t); }

cudaError_t exclusive_scan(const uint8_t* keep, int n, uint32_t* rank, uint32_t* tiles, cudaStream_t s) {
  const int nt = nblk_of((size_t)n, kMgThreads);
  scan_tiles_kernel<<<nt, kMgThreads, 0, s>>>(keep, n, rank, tiles);
  scan_sums_kernel<<<1, kMgThreads, 0, s>>>(tiles, nt);
  scan_add_kernel<<<nt, kMgThreads, 0, s>>>(rank, n, tiles);
  return cudaGetLastError();  // total at tiles[nt]
}

// stable sort of keys[0..n) (result in *keys; *other is scratch)
cudaError_t sort_keys(uint64_t** keys, uint64_t** other, int n, MgWork& w, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  key_bits_kernel<<<1, kMgThreads, 0, s>>>(*keys, n, w.bits);
  uint64_t hb[2];
  cudaError_t e = cudaMemcpyAsync(hb, w.bits, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const uint64_t vary = hb[0] & ~hb[1];
  const int nt = nblk_of((size_t)n, kMgThreads);
  for (int b = 0; b < 64; ++b) {
    if (!((vary >> b) & 1ull)) continue;
    bit_kernel<<<nt, kMgThreads, 0, s>>>(*keys, n, b, w.f8);
    if ((e = exclusive_scan(w.f8, n, w.rank, w.tiles, s)) != cudaSuccess) return e;
    split_scatter_kernel<<<nt, kMgThreads, 0, s>>>(*keys, n, w.f8, w.rank, w.tiles + nt, *other);
    std::swap(*keys, *other);
  }
  return cudaGetLastError();
}

// sorted, deduplicated (and, with lvl, not in the level) keys -> coordinates;
// returns the count through *count (host)
cudaError_t finish_list(uint64_t** keys, uint64_t** other, int n, const uint64_t* lvl, int nl, int32_t* out,
                        int* count, MgWork& w, cudaStream_t s) {
  *count = 0;
  if (n == 0) return cudaSuccess;
  cudaError_t e = sort_keys(keys, other, n, w, s);
  if (e != cudaSuccess) return e;
  const int nt = nblk_of((size_t)n, kMgThreads);
  select_kernel<<<nt, kMgThreads, 0, s>>>(*keys, n, lvl, nl, w.f8);
  if ((e = exclusive_scan(w.f8, n, w.rank, w.tiles, s)) != cudaSuccess) return e;
  compact_decode_kernel<<<nt, kMgThreads, 0, s>>>(*keys, n, w.f8, w.rank, out);
  uint32_t c = 0;
  e = cudaMemcpyAsync(&c, w.tiles + nt, sizeof(c), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *count = (int)c;
  return e;
}

}  // namespace

template <typename R>
static cudaError_t refine_level(int N, const R* f, int nblk, const int32_t* coords, double rel, uint8_t* flags,
                                int32_t* children, int32_t* buffer, int* counts, cudaStream_t s) {
  const size_t nmax = (size_t)nblk * 26;
  MgWork w;
  std::vector<void*> owned;
  cudaError_t e = cudaSuccess;
  auto get = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) owned.push_back(*p);
  };
  R* bmax = nullptr;
  get((void**)&bmax, sizeof(R) * nblk);
  get((void**)&w.k0, sizeof(uint64_t) * nmax);
  get((void**)&w.k1, sizeof(uint64_t) * nmax);
  get((void**)&w.lvl, sizeof(uint64_t) * nblk);
  get((void**)&w.bits, sizeof(uint64_t) * 2);
  get((void**)&w.f8, nmax);
  get((void**)&w.rank, sizeof(uint32_t) * nmax);
  get((void**)&w.tiles, sizeof(uint32_t) * (nblk_of(nmax, kMgThreads) + 1));
  get((void**)&w.cnt, sizeof(uint32_t) * 2);
  uint32_t nflag = 0;
  if (e == cudaSuccess) {
    uint32_t bad = 0;
    e = cudaMemsetAsync(w.cnt + 1, 0, sizeof(uint32_t), s);
    check_coords_kernel<<<nblk_of((size_t)3 * nblk, 256), 256, 0, s>>>(coords, nblk, w.cnt + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, w.cnt + 1, sizeof(bad), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && bad) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) {
    const int nb = nblk_of((size_t)nblk, kMgThreads);
    block_absmax_kernel<R><<<nblk, 256, 0, s>>>(f, N * N * N, bmax);
    flag_kernel<R><<<1, kMgThreads, 0, s>>>(bmax, nblk, rel, flags, w.cnt);
    e = exclusive_scan(flags, nblk, w.rank, w.tiles, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nflag, w.cnt, sizeof(nflag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // children of the flagged blocks (distinct for distinct parents)
    if (e == cudaSuccess && nflag > 0) {
      emit_kernel<<<nb, kMgThreads, 0, s>>>(coords, flags, w.rank, nblk, 1, w.k0);
      e = finish_list(&w.k0, &w.k1, (int)(8 * nflag), nullptr, 0, children, &counts[0], w, s);
    } else {
      counts[0] = 0;
    }
    // the level's keys, sorted, then the neighbours missing from the level
    if (e == cudaSuccess && nflag > 0) {
      level_keys_kernel<<<nb, kMgThreads, 0, s>>>(coords, nblk, w.lvl);
      uint64_t* lvl = w.lvl;
      uint64_t* tmp = w.k1;
      e = sort_keys(&lvl, &tmp, nblk, w, s);
      if (e == cudaSuccess && lvl != w.lvl)
        e = cudaMemcpyAsync(w.lvl, lvl, sizeof(uint64_t) * nblk, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) {
        e = exclusive_scan(flags, nblk, w.rank, w.tiles, s);  // ranks again (the sorts reused the scratch)
        emit_kernel<<<nb, kMgThreads, 0, s>>>(coords, flags, w.rank, nblk, 0, w.k0);
        e = finish_list(&w.k0, &w.k1, (int)(26 * nflag), w.lvl, nblk, buffer, &counts[1], w, s);
      }
    } else {
      counts[1] = 0;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* p : owned) cudaFree(p);
  return e;
}

template cudaError_t refine_level<float>(int, const float*, int, const int32_t*, double, uint8_t*, int32_t*, int32_t*,
                                         int*, cudaStream_t);
template cudaError_t refine_level<double>(int, const double*, int, const int32_t*, double, uint8_t*, int32_t*,
                                          int32_t*, int*, cudaStream_t);

cudaError_t launch_refine_level(int N, int prec_fp64, const void* f, int nblk, const int32_t* coords, double rel,
                                uint8_t* flags, int32_t* children, int32_t* buffer, int* counts, cudaStream_t s) {
  if ((size_t)nblk * 26 > (size_t)kMgMaxKeys) return cudaErrorInvalidValue;
  return prec_fp64 ? refine_level<double>(N, (const double*)f, nblk, coords, rel, flags, children, buffer, counts, s)
                   : refine_level<float>(N, (const float*)f, nblk, coords, rel, flags, children, buffer, counts, s);
}

}  // namespace flgf
