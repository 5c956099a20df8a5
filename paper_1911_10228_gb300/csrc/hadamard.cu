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
// Parent groups: the host packs the parents that have targets, in spatial
// order, into groups of at most 128.  The group's "cells" are the neighbour
// parents that hold sources, in block order; child b of cell c sits in slot
// b * ncell + c (zero where the child is absent or no source), so the threads
// of a warp -- consecutive parents of a full tile -- read consecutive 16-byte
// vectors.  A table in shared memory gives, per parent and neighbour e, the
// cell (or none); the host orders a group's parents by their set of
// neighbours with sources (most first, equal sets together), so that where a
// warp's parents share the set its lanes skip the same absent neighbours
// instead of idling while other lanes work.  Parents without targets and
// cells without sources take no thread and no shared memory, so sparse meshes
// keep the threads busy.
//
// CTA = (group) x (cpc chunks of T frequencies), 256 threads: a thread is
// (parent slot, frequency group, chunk).  Groups with few parents take
// several chunks per CTA so every CTA keeps 8 warps busy.  Shared memory
// holds, per chunk, the group's source spectra ([chunk][frequency
// group][slot], filled through L2 only) and the 343 kernel spectra; each
// thread holds the 8 source spectra of one neighbour cell in registers and
// reads the 27 distinct offsets d of that cell once each.  On levels that
// exclude the near field the host gives e = 0 (all pairs near) no cell, and
// the remaining near offsets |d|_inf <= 1 have zero spectra in the table
// (set up that way for octree levels >= 1).
// Complex multiply-adds are written as four fused multiply-adds.
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace flgf {

template <typename R, int TT>
__global__ void __launch_bounds__(kHadThreads, 2) hadamard_kernel(const HadGroup* __restrict__ groups,
                                                                  const HadWork* __restrict__ work,
                                                                  const int* __restrict__ src_ids,
                                                                  const int* __restrict__ tgt_ids,
                                                                  const uint16_t* __restrict__ par_tab,
                                                                  const cplx<R>* __restrict__ spec,
                                                                  cplx<R>* __restrict__ acc, int spec_blocks,
                                                                  const cplx<R>* __restrict__ kspec, size_t kstride) {
  constexpr int T = ChunkT<R>::value;
  constexpr int NG = T / TT;  // frequency groups per chunk
  static_assert(TT * sizeof(cplx<R>) == 16, "one 16-byte vector per (group, slot)");
  // [cpc][NG][8][ncell] source vectors, [cpc][343][T] kernel spectra, [27][nact] neighbour cells
  extern __shared__ __align__(16) int4 Fs[];
  const HadWork wk = work[blockIdx.x];
  const HadGroup gp = groups[wk.group];
  const int tid = threadIdx.x;
  const int NC = gp.ncell;
  const int S = 8 * NC;  // slots per (chunk, group): child b of cell c at b * NC + c

  int4* Ks = Fs + (size_t)gp.cpc * NG * S;
  // FP64 uses the three-product form (see below): per (offset, group) 32 bytes
  // holding kr, kr + ki, ki - kr and padding; FP32 keeps the complex values
  constexpr bool G3 = sizeof(R) == 8;
  constexpr int KV = (G3 ? 2 * kNOff * NG : kNOff * T * (int)sizeof(cplx<R>) / 16);  // 16-byte vectors per chunk
  uint16_t* NB = reinterpret_cast<uint16_t*>(Ks + (size_t)gp.cpc * KV);
  for (int i = tid; i < 27 * gp.nact; i += kHadThreads) NB[i] = par_tab[gp.par_off + i];
  if constexpr (G3) {
    for (int i = tid; i < wk.nch * kNOff * T; i += kHadThreads) {
      const int cs = i / (kNOff * T), d = (i / T) % kNOff, f = i % T;
      const cplx<R> k = kspec[(size_t)gp.level * kstride + ((size_t)(wk.chunk0 + cs) * kNOff + d) * T + f];
      R* dst = reinterpret_cast<R*>(Ks + (size_t)cs * KV + (size_t)(d * NG + f) * 2);
      dst[0] = k.re;
      dst[1] = k.re + k.im;
      dst[2] = k.im - k.re;
      dst[3] = R(0);
    }
  } else {
    for (int i = tid; i < wk.nch * KV; i += kHadThreads) {
      const int cs = i / KV, v = i % KV;
      Ks[i] = __ldg(reinterpret_cast<const int4*>(kspec + (size_t)gp.level * kstride + (size_t)(wk.chunk0 + cs) * kNOff * T) + v);
    }
  }
  for (int cs = 0; cs < wk.nch; ++cs) {
    int4* fdst = Fs + (size_t)cs * NG * S;
    for (int i = tid; i < S * NG; i += kHadThreads) {
      const int slot = i / NG, g = i % NG;
      const int sid = src_ids[gp.src_off + slot];
      fdst[g * S + slot] =
          sid >= 0 ? __ldcg(reinterpret_cast<const int4*>(spec + chunk_offset<R>(wk.chunk0 + cs, sid, spec_blocks)) + g)
                   : make_int4(0, 0, 0, 0);
    }
  }
  __syncthreads();

  const int slot = tid % gp.pslots;
  const int g = (tid / gp.pslots) % NG;
  const int cs = tid / (gp.pslots * NG);
  if (slot >= gp.nact || cs >= wk.nch) return;
  const int chunk = wk.chunk0 + cs;
  const int f0 = g * TT;
  const cplx<R>* Fg = reinterpret_cast<const cplx<R>*>(Fs + (size_t)(cs * NG + g) * S);
  const cplx<R>* Kc = reinterpret_cast<const cplx<R>*>(Ks + (size_t)cs * KV) + f0;  // complex form
  const int4* Kg = Ks + (size_t)cs * KV + g * 2;                                      // three-product form

  // FP32: ar, ai accumulate re and im with four FMAs per pair.  FP64 (bound by
  // the FP64 FMA rate) takes the three-product form: with s = fr + fi,
  // re(k f) = kr s - (kr + ki) fi and im(k f) = kr s + (ki - kr) fr, so the
  // accumulators ar = sum kr s, ai = sum (kr + ki) fi, a3 = sum (ki - kr) fr
  // take three FMAs per pair, and re = ar - ai, im = ar + a3.
  R ar[8][TT], ai[8][TT], a3[8][G3 ? TT : 1];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      ar[a][t] = R(0); ai[a][t] = R(0);
      if constexpr (G3) a3[a][t] = R(0);
    }

  // e stays the (warp-uniform) loop index, so the kernel-spectrum addresses
  // below are uniform across the warp; the next neighbour's cell is read one
  // iteration ahead
  unsigned cn = NB[slot];
  for (int e = 0; e < 27; ++e) {
    const unsigned cw = cn;
    if (e + 1 < 27) cn = NB[(e + 1) * gp.nact + slot];
    if (cw == kNbEnd) continue;  // no neighbour parent with sources (or e = 0 without near field)
    const int c = (int)cw;
    const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
    // the 8 children b of neighbour parent p + e, TT frequencies each (zero where absent)
    const cplx<R>* fb = Fg + (size_t)c * TT;
    R fr[8][TT], fi[8][TT], fs[8][G3 ? TT : 1];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const cplx<R> v = fb[(size_t)b * NC * TT + t];
        fr[b][t] = v.re; fi[b][t] = v.im;
        if constexpr (G3) fs[b][t] = v.re + v.im;
      }
    // d = a - b - 2e takes 27 values delta - 2e (delta = a - b in {-1,0,1}^3):
    // one kernel-spectrum load per delta, applied to every (a, b) pair with a - b = delta
    const int eoff = off_index(-2 * e0, -2 * e1, -2 * e2);
#pragma unroll
    for (int dl = 0; dl < 27; ++dl) {
      const int l0 = dl / 9 - 1, l1 = (dl / 3) % 3 - 1, l2 = dl % 3 - 1;
      const int d = eoff + l0 * 49 + l1 * 7 + l2;
      if constexpr (G3) {
        const int4* kp = Kg + (size_t)d * NG * 2;
        const int4 kv0 = kp[0], kv1 = kp[1];
        const R k0 = reinterpret_cast<const R*>(&kv0)[0], k1 = reinterpret_cast<const R*>(&kv0)[1];
        const R k2 = reinterpret_cast<const R*>(&kv1)[0];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int b0 = (a >> 2) - l0, b1 = ((a >> 1) & 1) - l1, b2 = (a & 1) - l2;
          if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b2 < 0 || b2 > 1) continue;  // resolved at compile time
          const int b = (b0 << 2) | (b1 << 1) | b2;
          ar[a][0] = fma(k0, fs[b][0], ar[a][0]);
          ai[a][0] = fma(k1, fi[b][0], ai[a][0]);
          a3[a][0] = fma(k2, fr[b][0], a3[a][0]);
        }
      } else {
        const int4 kv = *reinterpret_cast<const int4*>(Kc + (size_t)d * T);
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
  }
  // write the parent's targets
  const int* tg = tgt_ids + gp.tgt_off + slot * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int sid = __ldg(tg + a);
    if (sid < 0) continue;
    cplx<R>* o = acc + chunk_offset<R>(chunk, sid, spec_blocks) + f0;
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      if constexpr (G3) o[t] = cplx<R>{ar[a][t] - ai[a][t], ar[a][t] + a3[a][t]};
      else o[t] = cplx<R>{ar[a][t], ai[a][t]};
    }
  }
}

template <typename R>
cudaError_t launch_hadamard(int N, const HadGroup* groups, const HadWork* work, int nwork, int max_units,
                            const int* src_ids, const int* tgt_ids, const uint16_t* par_tab, const void* spec, void* acc,
                            int spec_blocks, const void* kspec, size_t kspec_level_stride, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  constexpr int TT = (sizeof(R) == 4) ? 2 : 1;
  // per chunk the group's source spectra and the 343 kernel spectra, and the
  // neighbour table: max_units 32-byte units
  const size_t sm = 32 * (size_t)max_units;
  if (sm > kHadSmemBytes) return cudaErrorInvalidConfiguration;
  // per device and cheap, so set on every launch (two CTAs per SM)
  cudaError_t e = cudaFuncSetAttribute(hadamard_kernel<R, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kHadSmemBytes);
  if (e != cudaSuccess) return e;
  hadamard_kernel<R, TT><<<nwork, kHadThreads, sm, s>>>(groups, work, src_ids, tgt_ids, par_tab,
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
  // the pair entries stream from global memory in batches of kPre, the next
  // batch in flight while the current one is multiplied (entries past the
  // list's end are zero: source slot 0, offset 0, not used)
  constexpr int kPre = 8;
  int wcur[kPre], wnxt[kPre];
#pragma unroll
  for (int q = 0; q < kPre; ++q) wnxt[q] = q < n ? __ldg(e + q * kListTargets) : 0;
  for (int j0 = 0; j0 < n; j0 += kPre) {
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      wcur[q] = wnxt[q];
      wnxt[q] = j0 + kPre + q < n ? __ldg(e + (j0 + kPre + q) * kListTargets) : 0;
    }
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      if (j0 + q >= n) break;
      const int w = wcur[q];
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
  cudaError_t e = cudaFuncSetAttribute(hadamard_list_kernel<R, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
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

template cudaError_t launch_hadamard<float>(int, const HadGroup*, const HadWork*, int, int, const int*, const int*,
                                            const uint16_t*, const void*, void*, int, const void*, size_t, cudaStream_t);
template cudaError_t launch_hadamard<double>(int, const HadGroup*, const HadWork*, int, int, const int*, const int*,
                                             const uint16_t*, const void*, void*, int, const void*, size_t, cudaStream_t);

// Shared memory of a group in 32-byte units: per chunk 8 slots per cell and
// the 343 kernel spectra, plus the [27][nact] int16 neighbour table.
static int group_units(int ncell, int nact, int cpc, int kunits) {
  return (8 * ncell + kunits) * cpc + (54 * nact + 31) / 32;
}

static int cell_key(const int* ch) {  // first child that is a source: identifies the cell
  for (int b = 0; b < 8; ++b)
    if (ch[b] >= 0) return ch[b];
  return -1;
}

void pack_parent_groups(int level, const std::vector<ParentRec>& recs, int nchunk, int kunits, HadLists& L,
                        bool order_by_list) {
  const int max_units = (int)(kHadSmemBytes / 32);
  size_t pos = 0;
  while (pos < recs.size()) {
    // take parents, in order, while the group's parents and cells fit
    std::unordered_map<int, int> cell_of;  // cell key -> index in `cells`
    std::vector<const int*> cells;         // the 8 children of each cell
    std::vector<size_t> members;
    while (pos < recs.size() && (int)members.size() < kHadMaxParents) {
      const ParentRec& r = recs[pos];
      int new_cells = 0;
      for (int e = 0; e < 27; ++e) {
        const int key = cell_key(r.cell[e]);
        new_cells += key >= 0 && !cell_of.count(key);
      }
      if (!members.empty() &&
          group_units((int)cells.size() + new_cells, (int)members.size() + 1, 1, kunits) > max_units)
        break;
      for (int e = 0; e < 27; ++e) {
        const int key = cell_key(r.cell[e]);
        if (key >= 0 && !cell_of.count(key)) {
          cell_of.emplace(key, (int)cells.size());
          cells.push_back(r.cell[e]);
        }
      }
      members.push_back(pos++);
    }
    // cells in block-id order (block ids follow the level's coordinate order on
    // the meshes built here), so that consecutive parents of a full tile see
    // consecutive cells and the warp's shared-memory reads do not conflict
    std::vector<int> order(cells.size());
    for (size_t c = 0; c < order.size(); ++c) order[c] = (int)c;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cell_key(cells[a]) < cell_key(cells[b]); });
    std::vector<const int*> sorted(cells.size());
    for (size_t c = 0; c < order.size(); ++c) {
      sorted[c] = cells[order[c]];
      cell_of[cell_key(sorted[c])] = (int)c;
    }
    cells.swap(sorted);

    // parents with equal neighbour sets side by side, largest sets first
    // (stable: spatial order within a class), so warps skip uniformly
    if (order_by_list) {
      auto mask = [&](size_t m) {
        uint32_t v = 0;
        for (int e = 0; e < 27; ++e) v |= (uint32_t)(cell_key(recs[m].cell[e]) >= 0) << e;
        return v;
      };
      std::vector<std::pair<uint32_t, size_t>> key(members.size());
      for (size_t i = 0; i < members.size(); ++i) key[i] = {mask(members[i]), members[i]};
      std::stable_sort(key.begin(), key.end(), [](const auto& x, const auto& y) {
        const int cx = __builtin_popcount(x.first), cy = __builtin_popcount(y.first);
        return cx != cy ? cx > cy : x.first < y.first;
      });
      for (size_t i = 0; i < members.size(); ++i) members[i] = key[i].second;
    }
    HadGroup gp;
    gp.level = level;
    gp.nact = (int)members.size();
    gp.ncell = (int)cells.size();
    gp.pslots = 1;
    while (gp.pslots < gp.nact) gp.pslots <<= 1;
    int cpc = std::min(kHadMaxCpc, kHadThreads / (gp.pslots * 2));
    while (cpc > 1 && group_units(gp.ncell, gp.nact, cpc, kunits) > max_units) cpc >>= 1;
    gp.cpc = cpc;
    L.max_units = std::max(L.max_units, group_units(gp.ncell, gp.nact, cpc, kunits));
    // sources: child b of cell c at slot b * ncell + c (-1: absent, zero spectrum)
    gp.src_off = (int)L.src_ids.size();
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < gp.ncell; ++c) L.src_ids.push_back(cells[c][b]);
    // per parent: the cell of each neighbour (e-major table, kNbEnd where the
    // neighbour has no sources) and the 8 targets
    gp.par_off = (int)L.par_tab.size();
    L.par_tab.resize(L.par_tab.size() + (size_t)27 * gp.nact, kNbEnd);
    gp.tgt_off = (int)L.tgt_ids.size();
    for (int m = 0; m < gp.nact; ++m) {
      const ParentRec& r = recs[members[m]];
      for (int e = 0; e < 27; ++e) {
        const int key = cell_key(r.cell[e]);
        if (key >= 0) L.par_tab[gp.par_off + e * gp.nact + m] = (uint16_t)cell_of.at(key);
      }
      L.tgt_ids.insert(L.tgt_ids.end(), r.tgt, r.tgt + 8);
    }
    for (int c0 = 0; c0 < nchunk; c0 += cpc)
      L.work.push_back(HadWork{(int)L.groups.size(), c0, std::min(cpc, nchunk - c0)});
    L.groups.push_back(gp);
  }
}

}  // namespace flgf
