// a3: spectrum multiply-accumulate over the interaction lists (Sec. 2.1,
// level interaction: v~_i = sum_{j in I(B_i)} conv(G_{i-j}, f~_j), each conv a
// Hadamard product of zero-padded spectra).
//
// Structure exploited: on octree level k the sources that interact with a
// target t are the children of the neighbours of t's parent (minus t's near
// neighbours on levels above the finest; on the top level this is every
// non-neighbour).  So the 8 children a of one parent p see the same 216
// source blocks 2(p + e) + b (e in {-1,0,1}^3, b in {0,1}^3), with kernel
// offset d = a - b - 2e.  One thread owns the 8 targets of a parent for TT
// frequencies; each source spectrum value it loads from shared memory is
// used 8 times, and the kernel spectra (indexed by d only) are the same for
// every thread of a warp (shared-memory broadcast).
//
// CTA = (tile of parents) x (cpc chunks of T frequencies), 256 threads: a
// thread is (parent slot, frequency group, chunk).  Tiles of the coarse
// octree levels have few parents and take several chunks per CTA so every
// CTA keeps 8 warps busy.  Shared memory holds, per chunk, the spectra of
// every source block in the tile's region (tile grown by one parent on each
// side, clipped to the level's bounding box; absent blocks are zero), stored
// parity-major -- [chunk][frequency group][child position b][parent cell q]
// -- so the threads of a warp (consecutive parents) read consecutive 16-byte
// vectors.  The host orders each tile's source list in that order, so the
// fill is a straight copy (through L2 only).  The CTA's kernel-spectrum
// chunks are staged in shared memory too: within a warp every thread needs
// the same offset d, so each read is one broadcast; per neighbour parent e
// the 27 distinct offsets are read once each and the 8 source spectra are
// held in registers.  On
// levels that exclude the near field, e = 0 (all pairs near) is skipped and
// the remaining near offsets |d|_inf <= 1 have zero spectra in the table
// (set up that way for octree levels >= 1).
// Complex multiply-adds are written as four fused multiply-adds.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace flgf {

template <typename R, int TT>
__global__ void __launch_bounds__(kHadThreads, 2) hadamard_kernel(const HadTile* __restrict__ tiles,
                                                                  const HadWork* __restrict__ work,
                                                                  const int* __restrict__ src_ids,
                                                                  const int* __restrict__ tgt_ids,
                                                                  const int2* __restrict__ pmap,
                                                                  const cplx<R>* __restrict__ spec,
                                                                  cplx<R>* __restrict__ acc, int spec_blocks,
                                                                  const cplx<R>* __restrict__ kspec, size_t kstride) {
  constexpr int T = ChunkT<R>::value;
  constexpr int NG = T / TT;  // frequency groups per chunk
  static_assert(TT * sizeof(cplx<R>) == 16, "one 16-byte vector per (group, cell)");
  extern __shared__ __align__(16) int4 Fs[];  // [cpc][NG][8 NQ] 16-byte vectors, then [cpc][343][T] kernel spectra
  const HadWork wk = work[blockIdx.x];
  const HadTile tl = tiles[wk.tile];
  const int tid = threadIdx.x;
  const int R1 = tl.Rg[1], R2 = tl.Rg[2];
  const int NQ = tl.Rg[0] * R1 * R2;
  const int S = 8 * NQ;  // slots per (chunk, group)

  // this CTA's kernel-spectrum chunks (343 x 32 bytes each) after the source region
  int4* Ks = Fs + (size_t)tl.cpc * NG * S;
  constexpr int KV = kNOff * T * (int)sizeof(cplx<R>) / 16;  // 16-byte vectors per chunk
  for (int i = tid; i < wk.nch * KV; i += kHadThreads) {
    const int cs = i / KV, v = i % KV;
    Ks[i] = __ldg(reinterpret_cast<const int4*>(kspec + (size_t)tl.level * kstride + (size_t)(wk.chunk0 + cs) * kNOff * T) + v);
  }
  for (int cs = 0; cs < wk.nch; ++cs) {
    int4* fdst = Fs + (size_t)cs * NG * S;
    for (int i = tid; i < S * NG; i += kHadThreads) {
      const int slot = i / NG, g = i % NG;
      const int sid = src_ids[tl.src_off + slot];
      fdst[g * S + slot] =
          sid >= 0 ? __ldcg(reinterpret_cast<const int4*>(spec + chunk_offset<R>(wk.chunk0 + cs, sid, spec_blocks)) + g)
                   : make_int4(0, 0, 0, 0);
    }
  }
  __syncthreads();

  const int slot = tid % tl.pslots;
  const int g = (tid / tl.pslots) % NG;
  const int cs = tid / (tl.pslots * NG);
  const int np = tl.P[0] * tl.P[1] * tl.P[2];
  if (slot >= np || cs >= wk.nch) return;
  const int2 pm = pmap[tl.pmap_off + slot];
  const int pl = pm.x;          // parent index in the tile
  const unsigned emask = pm.y;  // neighbours e that hold sources
  const int chunk = wk.chunk0 + cs;
  const int f0 = g * TT;
  const int pq[3] = {pl / (tl.P[1] * tl.P[2]), (pl / tl.P[2]) % tl.P[1], pl % tl.P[2]};
  const int q0 = tl.p0[0] + pq[0] - tl.r0[0], q1 = tl.p0[1] + pq[1] - tl.r0[1], q2 = tl.p0[2] + pq[2] - tl.r0[2];
  const cplx<R>* Fg = reinterpret_cast<const cplx<R>*>(Fs + (size_t)(cs * NG + g) * S);
  const cplx<R>* Kc = reinterpret_cast<const cplx<R>*>(Ks + (size_t)cs * KV) + f0;

  R ar[8][TT], ai[8][TT];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int t = 0; t < TT; ++t) { ar[a][t] = R(0); ai[a][t] = R(0); }

  for (int e = 0; e < 27; ++e) {
    if (!((emask >> e) & 1u)) continue;  // outside the region, no sources, or e = 0 without near field
    const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
    const int n0 = q0 + e0, n1 = q1 + e1, n2 = q2 + e2;
    // the 8 children b of neighbour parent p + e, TT frequencies each
    const cplx<R>* fb = Fg + (size_t)((n0 * R1 + n1) * R2 + n2) * TT;
    R fr[8][TT], fi[8][TT];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const cplx<R> v = fb[(size_t)b * NQ * TT + t];
        fr[b][t] = v.re; fi[b][t] = v.im;
      }
    // d = a - b - 2e takes 27 values delta - 2e (delta = a - b in {-1,0,1}^3):
    // one kernel-spectrum load per delta, applied to every (a, b) pair with a - b = delta
    const cplx<R>* kb = Kc + (size_t)off_index(-2 * e0, -2 * e1, -2 * e2) * T;
#pragma unroll
    for (int dl = 0; dl < 27; ++dl) {
      const int l0 = dl / 9 - 1, l1 = (dl / 3) % 3 - 1, l2 = dl % 3 - 1;
      const int4 kv = *reinterpret_cast<const int4*>(kb + (l0 * 49 + l1 * 7 + l2) * T);
      const cplx<R>* kk = reinterpret_cast<const cplx<R>*>(&kv);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int b0 = (a >> 2) - l0, b1 = ((a >> 1) & 1) - l1, b2 = (a & 1) - l2;
        if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b2 < 0 || b2 > 1) continue;  // resolved at compile time
        const int b = (b0 << 2) | (b1 << 1) | b2;
#pragma unroll
        for (int t = 0; t < TT; ++t) {
          const cplx<R> k = kk[t];
          ar[a][t] = fma(k.re, fr[b][t], ar[a][t]);
          ar[a][t] = fma(-k.im, fi[b][t], ar[a][t]);
          ai[a][t] = fma(k.re, fi[b][t], ai[a][t]);
          ai[a][t] = fma(k.im, fr[b][t], ai[a][t]);
        }
      }
    }
  }
  // write the 8 targets
  const int TP1 = 2 * tl.P[1], TP2 = 2 * tl.P[2];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int a0 = a >> 2, a1 = (a >> 1) & 1, a2 = a & 1;
    const int cell = ((2 * pq[0] + a0) * TP1 + (2 * pq[1] + a1)) * TP2 + (2 * pq[2] + a2);
    const int sid = tgt_ids[tl.tgt_off + cell];
    if (sid < 0) continue;
    cplx<R>* o = acc + chunk_offset<R>(chunk, sid, spec_blocks) + f0;
#pragma unroll
    for (int t = 0; t < TT; ++t) o[t] = cplx<R>{ar[a][t], ai[a][t]};
  }
}

template <typename R>
cudaError_t launch_hadamard(int N, const HadTile* tiles, const HadWork* work, int nwork, int max_cells_x_cpc,
                            const int* src_ids, const int* tgt_ids, const int2* pmap, const void* spec, void* acc,
                            int spec_blocks, const void* kspec, size_t kspec_level_stride, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  constexpr int T = ChunkT<R>::value;
  constexpr int TT = (sizeof(R) == 4) ? 2 : 1;
  // per chunk: the source region cells and the 343 kernel spectra (32 bytes each)
  const size_t sm = sizeof(cplx<R>) * T * (size_t)max_cells_x_cpc;
  if (sm > 110 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set[2] = {false, false};
  bool& done = attr_set[sizeof(R) == 4 ? 0 : 1];
  if (!done) {
    // two CTAs per SM need <= 2 x 110 KB of shared memory
    cudaError_t e = cudaFuncSetAttribute(hadamard_kernel<R, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024);
    if (e != cudaSuccess) return e;
    done = true;
  }
  hadamard_kernel<R, TT><<<nwork, kHadThreads, sm, s>>>(tiles, work, src_ids, tgt_ids, pmap,
                                                       reinterpret_cast<const cplx<R>*>(spec),
                                                       reinterpret_cast<cplx<R>*>(acc), spec_blocks,
                                                       reinterpret_cast<const cplx<R>*>(kspec), kspec_level_stride);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sparse tiles: each thread walks the explicit pair list of one target for TT
// frequencies.  Shared memory holds this chunk of the 343 kernel spectra and
// of the group's sources, so the loop reads only shared memory.
// ---------------------------------------------------------------------------
template <typename R, int TT>
__global__ void __launch_bounds__(kListTargets * 2) hadamard_list_kernel(const ListGroup* __restrict__ groups,
                                                                       const int* __restrict__ tgt,
                                                                       const int* __restrict__ len,
                                                                       const int* __restrict__ ent,
                                                                       const int* __restrict__ src,
                                                                       const cplx<R>* __restrict__ spec,
                                                                       cplx<R>* __restrict__ acc, int spec_blocks,
                                                                       const cplx<R>* __restrict__ kspec,
                                                                       size_t kstride) {
  constexpr int T = ChunkT<R>::value;
  constexpr int NG = T / TT;
  static_assert(NG == 2, "two frequency groups per chunk");
  extern __shared__ __align__(16) int4 sm4[];
  const ListGroup gr = groups[blockIdx.x];
  const int chunk = blockIdx.y;
  const int tid = threadIdx.x;
  constexpr int KV = kNOff * T * (int)sizeof(cplx<R>) / 16;  // 16-byte vectors of one kernel chunk
  // frequency-group-major ([NG][343], [NG][nsrc]): the lanes of a warp share
  // g, so their 16-byte reads spread over all eight bank groups
  int4* Ks = sm4;
  int4* Fs = sm4 + KV;
  const int4* kc = reinterpret_cast<const int4*>(kspec + (size_t)gr.level * kstride + (size_t)chunk * kNOff * T);
  for (int i = tid; i < KV; i += blockDim.x) Ks[(i % NG) * kNOff + i / NG] = __ldg(kc + i);
  for (int i = tid; i < gr.nsrc * NG; i += blockDim.x)
    Fs[(i % NG) * gr.nsrc + i / NG] =
        __ldcg(reinterpret_cast<const int4*>(spec + chunk_offset<R>(chunk, src[gr.src_off + i / NG], spec_blocks)) + i % NG);
  __syncthreads();
  const int ti = tid % kListTargets, g = tid / kListTargets;
  if (ti >= gr.ntgt) return;
  const int n = len[gr.len_off + ti];
  const int* e = ent + gr.ent_off + ti;
  R ar[TT], ai[TT];
#pragma unroll
  for (int t = 0; t < TT; ++t) { ar[t] = R(0); ai[t] = R(0); }
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    const int w = __ldg(e + j * kListTargets);
    const int4 fv = Fs[g * gr.nsrc + (w >> 9)];
    const int4 kv = Ks[g * kNOff + (w & 511)];
    const cplx<R>* f = reinterpret_cast<const cplx<R>*>(&fv);
    const cplx<R>* k = reinterpret_cast<const cplx<R>*>(&kv);
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      ar[t] = fma(k[t].re, f[t].re, ar[t]);
      ar[t] = fma(-k[t].im, f[t].im, ar[t]);
      ai[t] = fma(k[t].re, f[t].im, ai[t]);
      ai[t] = fma(k[t].im, f[t].re, ai[t]);
    }
  }
  cplx<R>* o = acc + chunk_offset<R>(chunk, tgt[gr.tgt_off + ti], spec_blocks) + g * TT;
#pragma unroll
  for (int t = 0; t < TT; ++t) o[t] = cplx<R>{ar[t], ai[t]};
}

template <typename R>
cudaError_t launch_hadamard_list(int N, const ListGroup* groups, int ngroups, int max_src, const int* tgt,
                                 const int* len, const int* ent, const int* src, const void* spec, void* acc,
                                 int spec_blocks, const void* kspec, size_t kspec_level_stride, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  constexpr int T = ChunkT<R>::value;
  constexpr int TT = (sizeof(R) == 4) ? 2 : 1;
  const size_t sm = sizeof(cplx<R>) * T * ((size_t)kNOff + max_src);
  if (sm > 200 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set[2] = {false, false};
  bool& done = attr_set[sizeof(R) == 4 ? 0 : 1];
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(hadamard_list_kernel<R, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    done = true;
  }
  dim3 grid(ngroups, nchunks<R>(N));
  hadamard_list_kernel<R, TT><<<grid, kListTargets * 2, sm, s>>>(
      groups, tgt, len, ent, src, reinterpret_cast<const cplx<R>*>(spec), reinterpret_cast<cplx<R>*>(acc),
      spec_blocks, reinterpret_cast<const cplx<R>*>(kspec), kspec_level_stride);
  return cudaGetLastError();
}

template cudaError_t launch_hadamard_list<float>(int, const ListGroup*, int, int, const int*, const int*, const int*,
                                                 const int*, const void*, void*, int, const void*, size_t,
                                                 cudaStream_t);
template cudaError_t launch_hadamard_list<double>(int, const ListGroup*, int, int, const int*, const int*,
                                                  const int*, const int*, const void*, void*, int, const void*,
                                                  size_t, cudaStream_t);

template cudaError_t launch_hadamard<float>(int, const HadTile*, const HadWork*, int, int, const int*, const int*,
                                            const int2*, const void*, void*, int, const void*, size_t, cudaStream_t);
template cudaError_t launch_hadamard<double>(int, const HadTile*, const HadWork*, int, int, const int*, const int*,
                                             const int2*, const void*, void*, int, const void*, size_t, cudaStream_t);

void build_parent_map(const HadTile& tl, const int* src_slots, const int* tgt_slots, std::vector<int2>& out) {
  const int np = tl.P[0] * tl.P[1] * tl.P[2];
  const int NQ = tl.Rg[0] * tl.Rg[1] * tl.Rg[2];
  std::vector<int2> m(np);
  for (int pl = 0; pl < np; ++pl) {
    const int pq[3] = {pl / (tl.P[1] * tl.P[2]), (pl / tl.P[2]) % tl.P[1], pl % tl.P[2]};
    unsigned mask = 0;
    bool has_tgt = false;  // a parent without targets does no work
    for (int a = 0; a < 8; ++a) {
      const int cell = ((2 * pq[0] + (a >> 2)) * 2 * tl.P[1] + (2 * pq[1] + ((a >> 1) & 1))) * 2 * tl.P[2] +
                       (2 * pq[2] + (a & 1));
      has_tgt |= tgt_slots[cell] >= 0;
    }
    if (!has_tgt) {
      m[pl] = make_int2(pl, 0);
      continue;
    }
    for (int e = 0; e < 27; ++e) {
      if (tl.excl_near && e == 13) continue;
      int n[3];
      bool in = true;
      for (int a = 0; a < 3; ++a) {
        const int ea = (a == 0 ? e / 9 : a == 1 ? (e / 3) % 3 : e % 3) - 1;
        n[a] = tl.p0[a] + pq[a] - tl.r0[a] + ea;
        in &= n[a] >= 0 && n[a] < tl.Rg[a];
      }
      if (!in) continue;
      const int q = (n[0] * tl.Rg[1] + n[1]) * tl.Rg[2] + n[2];
      bool any = false;
      for (int b = 0; b < 8; ++b) any |= src_slots[b * NQ + q] >= 0;
      if (any) mask |= 1u << e;
    }
    m[pl] = make_int2(pl, (int)mask);
  }
  // spatial order: consecutive threads read consecutive shared-memory vectors
  out.insert(out.end(), m.begin(), m.end());
}

}  // namespace flgf
