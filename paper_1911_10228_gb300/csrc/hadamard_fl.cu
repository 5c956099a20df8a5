// a3, FP32: the spectrum multiply-accumulate with one frequency per lane
// (Sec. 2.1, level interaction: each target block's spectrum collects
// K^_{t-s} (.) F^_s over its near and influence lists).
//
// Mapping.  A CTA takes a group of at most kFlMaxParents target parents (the
// parents whose children are targets) and a block of kFlFreq = 64
// consecutive frequencies; a warp owns one parent at a time and lane l holds
// frequencies 2l and 2l + 1 (16 bytes).  All lanes of a warp share the parent's list of
// neighbour cells with sources and the child masks (which of the parent's 8
// children are targets, which of a cell's 8 children are sources), so absent
// cells and children are skipped by warp-uniform control flow: no lane idles
// while another works.
//
// Memory.  Shared memory holds the 343 kernel spectra of the frequency block,
// [343][64] (176 KB): a kernel read is a row of 64 consecutive frequencies
// (conflict-free), and the group's tables (the spectrum columns of its cells'
// children, the parents' neighbour lists and targets).  The source spectra
// are read from global memory (L2, and L1 for cells shared by the CTA's
// parents): a cell child's 64 frequencies are four 128-byte lines of the
// chunked spectrum layout, one 16-byte load per lane, and the next cell's
// sources are in flight while the current one is multiplied.  One CTA of
// kFlWarps = 12 warps per SM.
//
// Per (parent, cell) the structure of the block-pair offsets is used as in
// the parent-group kernel: the 8 x 8 (target a, source b) pairs of the parent
// and the neighbour parent p + e take kernel offset d = (a - b) - 2e, so one
// kernel-spectrum read serves every pair with the same delta = a - b.  The
// host gives each (parent, cell) a 27-bit mask of the deltas that carry a
// product: some present target a and source b with that difference, and, on
// octree levels above the finest, a kernel offset outside the near range
// (|d| <= 1 there has a zero kernel spectrum).  A delta in the mask runs all
// its pairs unconditionally -- an absent source child was loaded as zero and
// an absent target's accumulator is never stored, so those products change
// nothing -- and a delta outside it is skipped by one warp-uniform branch.
// One straight-line path per delta keeps the unrolled code small (it stays
// in the instruction cache) and free of per-pair branches; the kernel read of
// the next delta is issued before the products of the current one.  Rows
// whose mask holds every delta (bit 31 set by the host; near deltas of a
// coarse level, whose kernel spectra are zero, count as held) need no tests at
// all: in phases where at least 90 % of the rows are full, the kernel runs
// those rows as one straight-line block (the two-path form, faster there),
// while phases with rows of both kinds keep the single path, whose code stays
// within the instruction cache.  Both forms compute the same products in the
// same order.
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace flgf {

namespace {

constexpr int kFlThreads = 32 * kFlWarps;

// shared-memory bytes of a group's tables: cell columns, targets, delta masks, rows
size_t fl_table_bytes(int max_cells, int max_parents) {
  return sizeof(int) * 8 * ((size_t)max_cells + max_parents) + sizeof(uint32_t) * (size_t)kFlDelta * max_parents +
         sizeof(uint16_t) * (size_t)kFlRowStride * max_parents;
}

// two frequencies: k, f hold (re, im) of frequency 0 in x, y and of frequency 1 in z, w
__device__ __forceinline__ void cmac(float (&ar)[2], float (&ai)[2], float4 k, float4 f) {
  ar[0] = fmaf(k.x, f.x, ar[0]);
  ar[0] = fmaf(-k.y, f.y, ar[0]);
  ai[0] = fmaf(k.x, f.y, ai[0]);
  ai[0] = fmaf(k.y, f.x, ai[0]);
  ar[1] = fmaf(k.z, f.z, ar[1]);
  ar[1] = fmaf(-k.w, f.w, ar[1]);
  ai[1] = fmaf(k.z, f.w, ai[1]);
  ai[1] = fmaf(k.w, f.z, ai[1]);
}

// The 8 children of a cell (their spectrum columns in shared memory) at this
// lane's frequency, zero where absent; returns the cell's source mask.  The
// lane's offset into the chunked spectrum layout is fixed (lane_spec), a
// source column adds 4 T complex values per column.
// The loads are volatile inline PTX so that the compiler issues them where
// they stand (one cell ahead of their use) instead of sinking them towards
// the products; a load is predicated off for an absent child (sid < 0), which
// keeps its zero.
__device__ __forceinline__ float4 ld_cg_f4_if(const float4* p, int sid) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ge.s32 q, %5, 0;\n\t@q ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];\n\t}"
      : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w)
      : "l"(p), "r"(sid));
  return v;
}
__device__ __forceinline__ void load_cell(const int* cid, const float2* __restrict__ lane_spec, float4 (&f)[8]) {
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int sid = cid[b];
    f[b] = ld_cg_f4_if(reinterpret_cast<const float4*>(lane_spec + (size_t)max(sid, 0) * (kChunkGroup * ChunkT<float>::value)),
                       sid);
  }
}

// The products of one (parent, cell): kernel offset d = (a - b) - 2e; Kc
// points at d = -2e, dlm is the row's delta mask.
// One path for every row: delta dl runs its pairs when its mask bit is set
// (every bit on full rows), and the kernel read of the next delta is issued,
// unconditionally, before the products of the current one, so that its
// shared-memory latency overlaps them.
__device__ __forceinline__ void cell_products_single(const float4* __restrict__ Kc, uint32_t dlm, const float4 (&f)[8],
                                                     float (&ar)[8][2], float (&ai)[8][2]) {
  if (dlm >> 31) dlm = (1u << 27) - 1;
  float4 kn = Kc[(-49 - 7 - 1) * (kFlFreq / 2)];
#pragma unroll
  for (int dl = 0; dl < 27; ++dl) {
    const float4 k = kn;
    if (dl + 1 < 27) {
      const int m0 = (dl + 1) / 9 - 1, m1 = ((dl + 1) / 3) % 3 - 1, m2 = (dl + 1) % 3 - 1;
      kn = Kc[(m0 * 49 + m1 * 7 + m2) * (kFlFreq / 2)];
    }
    if (!((dlm >> dl) & 1u)) continue;
    const int l0 = dl / 9 - 1, l1 = (dl / 3) % 3 - 1, l2 = dl % 3 - 1;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int b0 = (a >> 2) - l0, b1 = ((a >> 1) & 1) - l1, b2 = (a & 1) - l2;
      if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b2 < 0 || b2 > 1) continue;  // compile time
      cmac(ar[a], ai[a], k, f[(b0 << 2) | (b1 << 1) | b2]);
    }
  }
}

template <bool kAll>
__device__ __forceinline__ void cell_products_m(const float4* __restrict__ Kc, uint32_t dlm, const float4 (&f)[8],
                                                float (&ar)[8][2], float (&ai)[8][2]) {
#pragma unroll
  for (int dl = 0; dl < 27; ++dl) {
    if (!kAll && !((dlm >> dl) & 1u)) continue;
    const int l0 = dl / 9 - 1, l1 = (dl / 3) % 3 - 1, l2 = dl % 3 - 1;
    const float4 k = Kc[(l0 * 49 + l1 * 7 + l2) * (kFlFreq / 2)];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int b0 = (a >> 2) - l0, b1 = ((a >> 1) & 1) - l1, b2 = (a & 1) - l2;
      if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b2 < 0 || b2 > 1) continue;  // compile time
      cmac(ar[a], ai[a], k, f[(b0 << 2) | (b1 << 1) | b2]);
    }
  }
}
__device__ __forceinline__ void cell_products_split(const float4* __restrict__ Kc, uint32_t dlm, const float4 (&f)[8],
                                              float (&ar)[8][2], float (&ai)[8][2]) {
  if (dlm >> 31)
    cell_products_m<true>(Kc, dlm, f, ar, ai);
  else
    cell_products_m<false>(Kc, dlm, f, ar, ai);
}

// kSplit: the two-path form (phases whose rows are nearly all full), else the
// single path (its code stays within the instruction cache when rows of both
// kinds alternate).
template <bool kSplit>
__device__ __forceinline__ void cell_products(const float4* __restrict__ Kc, uint32_t dlm, const float4 (&f)[8],
                                              float (&ar)[8][2], float (&ai)[8][2]) {
  if constexpr (kSplit)
    cell_products_split(Kc, dlm, f, ar, ai);
  else
    cell_products_single(Kc, dlm, f, ar, ai);
}

__device__ __forceinline__ const float4* kernel_row(const float4* Ks, int w, int lane) {
  const int e = w >> 11;
  const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
  return Ks + off_index(-2 * e0, -2 * e1, -2 * e2) * (kFlFreq / 2) + lane;
}

}  // namespace

// kVec: a vector block set (ncomp components); the scalar form compiles
// without the component loop.
template <bool kVec, bool kSplit>
__global__ void __launch_bounds__(kFlThreads, 1)
    hadamard_fl_kernel(const FlGroup* __restrict__ groups, int ngroups, const uint16_t* __restrict__ rows,
                       const uint32_t* __restrict__ dlms, const int* __restrict__ tgt_ids, const int* __restrict__ cells,
                       const float2* __restrict__ spec, float2* __restrict__ acc, int spec_blocks,
                       const float2* __restrict__ kspec, size_t kstride, int ncomp, int cstride) {
  constexpr int T = ChunkT<float>::value;  // 4 frequencies per chunk
  constexpr int CPB = kFlFreq / T;         // 16 chunks per frequency block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ks = reinterpret_cast<float2*>(smem_raw);  // [343][64]
  const int id = blockIdx.x;
  const int g = id % ngroups, fb = id / ngroups;     // consecutive CTAs share the frequency block
  const FlGroup gp = groups[g];
  int* CI = reinterpret_cast<int*>(Ks + kNOff * kFlFreq);             // [ncell][8] spectrum columns
  int* TG = CI + gp.ncell * 8;                                         // [nact][8] targets
  uint32_t* DM = reinterpret_cast<uint32_t*>(TG + gp.nact * 8);       // [nact][kFlDelta] delta masks
  uint16_t* PR = reinterpret_cast<uint16_t*>(DM + gp.nact * kFlDelta); // [nact][kFlRowStride]
  const int tid = threadIdx.x;
  const int chunk0 = fb * CPB;

  // kernel spectra of the block: CPB chunks of [343][T], contiguous in the table
  {
    const int4* src = reinterpret_cast<const int4*>(kspec + (size_t)gp.level * kstride + (size_t)chunk0 * kNOff * T);
    constexpr int NV = CPB * kNOff * T / 2;  // 16-byte vectors (two complex values each)
    for (int i = tid; i < NV; i += kFlThreads) {
      const int4 v = __ldg(src + i);
      const int idx = 2 * i;                 // [chunk][d][t], t even
      const int c = idx / (kNOff * T), r = idx % (kNOff * T), d = r / T, t = r % T;
      float2* dst = Ks + d * kFlFreq + c * T + t;
      dst[0] = make_float2(__int_as_float(v.x), __int_as_float(v.y));
      dst[1] = make_float2(__int_as_float(v.z), __int_as_float(v.w));
    }
  }
  for (int i = tid; i < gp.ncell * 8; i += kFlThreads) CI[i] = __ldg(cells + (size_t)gp.cell_off * 8 + i);
  for (int i = tid; i < gp.nact * 8; i += kFlThreads) TG[i] = __ldg(tgt_ids + (size_t)gp.row_off * 8 + i);
  for (int i = tid; i < gp.nact * kFlDelta; i += kFlThreads) DM[i] = __ldg(dlms + (size_t)gp.row_off * kFlDelta + i);
  for (int i = tid; i < gp.nact * kFlRowStride; i += kFlThreads) PR[i] = __ldg(rows + (size_t)gp.row_off * kFlRowStride + i);
  __syncthreads();

  const int lane = tid & 31, warp = tid >> 5;
  const int chunk = chunk0 + (2 * lane) / T, t = (2 * lane) % T;  // this lane's two frequencies (t even)
  const float4* Ks4 = reinterpret_cast<const float4*>(Ks);
  // components of a vector block set: the same groups at columns + c cstride,
  // against the kernel spectra and tables staged once
  for (int comp = 0; comp < (kVec ? ncomp : 1); ++comp) {
  const size_t coff = (size_t)comp * cstride * (kChunkGroup * T);
  const float2* lane_spec = spec + chunk_offset<float>(chunk, 0, spec_blocks) + t + coff;
  float2* lane_acc = acc + chunk_offset<float>(chunk, 0, spec_blocks) + t + coff;
  for (int pm = warp; pm < gp.nact; pm += kFlWarps) {
    const uint16_t* row = PR + pm * kFlRowStride;
    const uint32_t* dm = DM + pm * kFlDelta;
    const int* tg = TG + pm * 8;
    const int ncl = row[0];
    float ar[8][2], ai[8][2];
#pragma unroll
    for (int a = 0; a < 8; ++a) { ar[a][0] = ar[a][1] = 0.f; ai[a][0] = ai[a][1] = 0.f; }
    // cells in pairs, ping-ponging two register buffers: the next cell's
    // sources are in flight while the current one is multiplied
    float4 fa[8], fb[8];
    if (ncl > 0) load_cell(CI + 8 * (row[1] & 0x7FF), lane_spec, fa);
    for (int j = 0; j < ncl; j += 2) {
      if (j + 1 < ncl) load_cell(CI + 8 * (row[2 + j] & 0x7FF), lane_spec, fb);
      cell_products<kSplit>(kernel_row(Ks4, row[1 + j], lane), dm[j], fa, ar, ai);
      if (j + 1 >= ncl) break;
      if (j + 2 < ncl) load_cell(CI + 8 * (row[3 + j] & 0x7FF), lane_spec, fa);
      cell_products<kSplit>(kernel_row(Ks4, row[2 + j], lane), dm[j + 1], fb, ar, ai);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (tg[a] < 0) continue;
      *reinterpret_cast<float4*>(lane_acc + (size_t)tg[a] * (kChunkGroup * T)) =
          make_float4(ar[a][0], ai[a][0], ar[a][1], ai[a][1]);
    }
  }
  }
}

namespace {
__device__ __forceinline__ void cmac1(float& ar, float& ai, float2 k, float2 f) {
  ar = fmaf(k.x, f.x, ar);
  ar = fmaf(-k.y, f.y, ar);
  ai = fmaf(k.x, f.y, ai);
  ai = fmaf(k.y, f.x, ai);
}
}  // namespace

// ---------------------------------------------------------------------------
// Pair lists in frequency lanes (the targets of sparse tiles, where few of a
// parent's 8 x 8 child pairs exist): a warp owns one target block and walks
// its (source, kernel offset) list; each lane holds one frequency of the
// CTA's 32-frequency block.  The list is read 32 entries at a time, one per
// lane, and broadcast by shuffles; eight source loads per warp are in flight
// before their products (sixteen, with 24 warps per CTA, measured 1 % slower
// on the batch, and so did L2 prefetches of the next entries' sources).  The
// kernel spectra of the block ([343][32], 88 KB) sit in shared
// memory, the sources come through L1 (the group's targets are spatially
// close and share most of them).  Per pair a lane reads 8 bytes of source and
// 8 of kernel for 4 FMAs: the unified L1/shared-memory data path bounds the
// kernel near a quarter of the FMA rate, against one eighth for the
// shared-memory pair-list kernel.  The products of a target run in list order
// into two accumulators (even and odd list positions), summed at the end.
// ---------------------------------------------------------------------------
namespace {
constexpr int kFllThreads = 32 * kFllWarps;
constexpr int kFllBatch = 8;  // source loads in flight per warp
}  // namespace

// U consecutive list entries of the lane-held batch starting at jj: U source
// loads in flight, then their products into the even / odd accumulators.
template <int U>
__device__ __forceinline__ void fll_batch(uint32_t my, int jj, const float2* __restrict__ lane_spec,
                                          const float2* __restrict__ Kl, float& ar0, float& ai0, float& ar1,
                                          float& ai1) {
  constexpr size_t kCol = kChunkGroup * ChunkT<float>::value;
  uint32_t e[U];
  float2 f[U];
#pragma unroll
  for (int u = 0; u < U; ++u) e[u] = __shfl_sync(0xffffffffu, my, jj + u);
#pragma unroll
  for (int u = 0; u < U; ++u) f[u] = __ldg(lane_spec + (size_t)(e[u] >> 9) * kCol);
#pragma unroll
  for (int u = 0; u < U; u += 2) {
    cmac1(ar0, ai0, Kl[(e[u] & 511u) * kFllFreq], f[u]);
    cmac1(ar1, ai1, Kl[(e[u + 1] & 511u) * kFllFreq], f[u + 1]);
  }
}

__global__ void __launch_bounds__(kFllThreads, 1)
    hadamard_fll_kernel(const FllGroup* __restrict__ groups, int ngroups, const int* __restrict__ tgt,
                        const int* __restrict__ beg, const int* __restrict__ len, const uint32_t* __restrict__ ent,
                        const float2* __restrict__ spec, float2* __restrict__ acc, int spec_blocks,
                        const float2* __restrict__ kspec, size_t kstride) {
  constexpr int T = ChunkT<float>::value;
  constexpr int CPB = kFllFreq / T;  // 8 chunks per frequency block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ks = reinterpret_cast<float2*>(smem_raw);  // [343][32]
  const int id = blockIdx.x;
  const int g = id % ngroups, fb = id / ngroups;
  const FllGroup gp = groups[g];
  const int tid = threadIdx.x;
  const int chunk0 = fb * CPB;
  {
    const int4* src = reinterpret_cast<const int4*>(kspec + (size_t)gp.level * kstride + (size_t)chunk0 * kNOff * T);
    constexpr int NV = CPB * kNOff * T / 2;
    for (int i = tid; i < NV; i += kFllThreads) {
      const int4 v = __ldg(src + i);
      const int idx = 2 * i;
      const int c = idx / (kNOff * T), r = idx % (kNOff * T), d = r / T, t = r % T;
      float2* dst = Ks + d * kFllFreq + c * T + t;
      dst[0] = make_float2(__int_as_float(v.x), __int_as_float(v.y));
      dst[1] = make_float2(__int_as_float(v.z), __int_as_float(v.w));
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int chunk = chunk0 + lane / T, t = lane % T;
  const float2* lane_spec = spec + chunk_offset<float>(chunk, 0, spec_blocks) + t;
  float2* lane_acc = acc + chunk_offset<float>(chunk, 0, spec_blocks) + t;
  const float2* Kl = Ks + lane;
  constexpr size_t kCol = kChunkGroup * T;  // complex values between two blocks' columns
  for (int m = warp; m < gp.ntgt; m += kFllWarps) {
    const int ti = gp.tgt_off + m;
    const int n = __ldg(len + ti), b0 = __ldg(beg + ti), tcol = __ldg(tgt + ti);
    float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
    for (int j0 = 0; j0 < n; j0 += 32) {
      const uint32_t my = j0 + lane < n ? __ldg(ent + b0 + j0 + lane) : 0u;
      const int cnt = min(32, n - j0);
      int jj = 0;
      for (; jj + kFllBatch <= cnt; jj += kFllBatch)
        fll_batch<kFllBatch>(my, jj, lane_spec, Kl, ar0, ai0, ar1, ai1);
      for (; jj < cnt; ++jj) {
        const uint32_t e = __shfl_sync(0xffffffffu, my, jj);
        cmac1(ar0, ai0, Kl[(e & 511u) * kFllFreq], __ldg(lane_spec + (size_t)(e >> 9) * kCol));
      }
    }
    lane_acc[(size_t)tcol * kCol] = make_float2(ar0 + ar1, ai0 + ai1);
  }
}

cudaError_t launch_hadamard_fll(int N, const FllGroup* groups, int ngroups, const int* tgt, const int* beg,
                                const int* len, const uint32_t* ent, const void* spec, void* acc, int spec_blocks,
                                const void* kspec, size_t kspec_level_stride, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  const int nfb = nfreq(N) / kFllFreq;
  const size_t sm = sizeof(float2) * (size_t)kNOff * kFllFreq;
  if ((size_t)nfb * ngroups >= (1u << 31)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(hadamard_fll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  hadamard_fll_kernel<<<(unsigned)(nfb * ngroups), kFllThreads, sm, s>>>(
      groups, ngroups, tgt, beg, len, ent, reinterpret_cast<const float2*>(spec), reinterpret_cast<float2*>(acc),
      spec_blocks, reinterpret_cast<const float2*>(kspec), kspec_level_stride);
  return cudaGetLastError();
}

size_t fl_smem_bytes(int max_cells, int max_parents) {
  return sizeof(float2) * (size_t)kNOff * kFlFreq + fl_table_bytes(max_cells, max_parents);
}

cudaError_t launch_hadamard_fl(int N, const FlGroup* groups, int ngroups, int max_cells, int max_parents,
                               const uint16_t* rows, const uint32_t* dlms, const int* tgt_ids, const int* cells,
                               const void* spec, void* acc, int spec_blocks, const void* kspec,
                               size_t kspec_level_stride, int ncomp, int cstride, bool split, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  if (ncomp < 1) return cudaErrorInvalidValue;
  const int nfb = nfreq(N) / kFlFreq;
  const size_t sm = fl_smem_bytes(max_cells, max_parents);
  if (sm > kFlSmemBytes || (size_t)nfb * ngroups >= (1u << 31)) return cudaErrorInvalidConfiguration;
  auto kern = ncomp > 1 ? (split ? hadamard_fl_kernel<true, true> : hadamard_fl_kernel<true, false>)
                        : (split ? hadamard_fl_kernel<false, true> : hadamard_fl_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(nfb * ngroups), kFlThreads, sm, s>>>(
      groups, ngroups, rows, dlms, tgt_ids, cells, reinterpret_cast<const float2*>(spec), reinterpret_cast<float2*>(acc),
      spec_blocks, reinterpret_cast<const float2*>(kspec), kspec_level_stride, ncomp, cstride);
  return cudaGetLastError();
}

// Bit delta (delta = a - b + (1, 1, 1) in base 3) of the (parent, neighbour e)
// products: some target child a and source child b with that difference,
// whose kernel offset d = delta - 2e is not a near offset of a coarse octree
// level (zero kernel spectrum there).  Bit 31: every delta is either held or
// such a near delta, so the row may run all 27 unconditionally.
uint32_t fl_delta_mask(int level, int e, const int* tgt, const int* src) {
  const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
  uint32_t mask = 0, near = 0;
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      const int l0 = (a >> 2) - (b >> 2), l1 = ((a >> 1) & 1) - ((b >> 1) & 1), l2 = (a & 1) - (b & 1);
      const int d0 = l0 - 2 * e0, d1 = l1 - 2 * e1, d2 = l2 - 2 * e2;
      const uint32_t bit = 1u << (((l0 + 1) * 3 + (l1 + 1)) * 3 + (l2 + 1));
      if (level > 0 && std::abs(d0) <= 1 && std::abs(d1) <= 1 && std::abs(d2) <= 1) {
        near |= bit;
        continue;
      }
      if (tgt[a] >= 0 && src[b] >= 0) mask |= bit;
    }
  if (mask && (mask | near) == (1u << 27) - 1) mask |= 1u << 31;
  return mask;
}

static int fl_cell_key(const int* ch) {
  for (int b = 0; b < 8; ++b)
    if (ch[b] >= 0) return ch[b];
  return -1;
}

void pack_fl_groups(int level, const std::vector<ParentRec>& recs, FlLists& L) {
  size_t pos = 0;
  while (pos < recs.size()) {
    // consecutive parents (tile order, so they share cells) while the group's cells fit
    std::unordered_map<int, int> cell_of;
    std::vector<const int*> cells;
    std::vector<size_t> members;
    while (pos < recs.size() && (int)members.size() < kFlMaxParents) {
      const ParentRec& r = recs[pos];
      int add = 0;
      for (int e = 0; e < 27; ++e) {
        const int key = fl_cell_key(r.cell[e]);
        add += key >= 0 && !cell_of.count(key);
      }
      if (!members.empty() && (int)cells.size() + add > kFlMaxCells) break;
      for (int e = 0; e < 27; ++e) {
        const int key = fl_cell_key(r.cell[e]);
        if (key >= 0 && !cell_of.count(key)) {
          cell_of.emplace(key, (int)cells.size());
          cells.push_back(r.cell[e]);
        }
      }
      members.push_back(pos++);
    }
    FlGroup gp;
    gp.level = level;
    gp.nact = (int)members.size();
    gp.ncell = (int)cells.size();
    gp.row_off = (int)(L.tgt_ids.size() / 8);
    gp.cell_off = (int)(L.cells.size() / 8);
    for (const int* ch : cells) L.cells.insert(L.cells.end(), ch, ch + 8);
    for (size_t m : members) {
      const ParentRec& r = recs[m];
      L.tgt_ids.insert(L.tgt_ids.end(), r.tgt, r.tgt + 8);
      std::vector<uint16_t> row(kFlRowStride, 0);
      std::vector<uint32_t> dm(kFlDelta, 0);
      int n = 0;
      for (int e = 0; e < 27; ++e) {
        const int key = fl_cell_key(r.cell[e]);
        if (key < 0) continue;
        const uint32_t mask = fl_delta_mask(level, e, r.tgt, r.cell[e]);
        if (!mask) continue;  // only near pairs of a coarse octree level: nothing to add
        dm[n] = mask;
        row[1 + n++] = (uint16_t)((e << 11) | cell_of.at(key));
      }
      row[0] = (uint16_t)n;
      L.rows.insert(L.rows.end(), row.begin(), row.end());
      L.dlms.insert(L.dlms.end(), dm.begin(), dm.end());
    }
    L.max_cells = std::max(L.max_cells, gp.ncell);
    L.max_parents = std::max(L.max_parents, gp.nact);
    L.groups.push_back(gp);
  }
}

void pack_fll_groups(int level, const std::vector<std::pair<int, std::vector<int>>>& pool, FllLists& L) {
  for (size_t pos = 0; pos < pool.size(); pos += kFllTargets) {
    const size_t end = std::min(pool.size(), pos + (size_t)kFllTargets);
    std::vector<size_t> members;
    for (size_t i = pos; i < end; ++i) members.push_back(i);
    // longest lists first: the warps' round-robin over targets stays balanced
    std::stable_sort(members.begin(), members.end(),
                     [&](size_t a, size_t b) { return pool[a].second.size() > pool[b].second.size(); });
    FllGroup g;
    g.level = level;
    g.ntgt = (int)members.size();
    g.tgt_off = (int)L.tgt.size();
    for (size_t m : members) {
      L.tgt.push_back(pool[m].first);
      L.beg.push_back((int)L.ent.size());
      L.len.push_back((int)pool[m].second.size());
      for (int w : pool[m].second) L.ent.push_back((uint32_t)w);
    }
    L.groups.push_back(g);
  }
}

}  // namespace flgf
