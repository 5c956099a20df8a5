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
// CTA = (tile of parents) x (one chunk of T frequencies).  Shared memory holds
// the chunk of the 343 kernel spectra of this octree level and the chunk of
// every source block in the tile's region (tile grown by one parent on each
// side, clipped to the level's bounding box; absent blocks are zero).  The
// region is stored parity-major, [freq group][child position b][parent cell
// q][TT], so the 32 threads of a warp (consecutive parents) read 32
// consecutive 16-byte vectors: no bank conflicts.  Near offsets |d|_inf <= 1
// are zeroed in shared memory on levels that exclude the near field, and
// e = 0 is skipped there entirely.  Complex multiply-adds are written as four
// fused multiply-adds.
#include "common.cuh"
#include "internal.h"

namespace flgf {

template <typename R, int TT>
__global__ void __launch_bounds__(256, 2) hadamard_kernel(const HadTile* __restrict__ tiles, const int* __restrict__ src_ids,
                                                          const int* __restrict__ tgt_ids, const cplx<R>* __restrict__ spec,
                                                          cplx<R>* __restrict__ acc, int spec_blocks,
                                                          const cplx<R>* __restrict__ kspec, size_t kstride) {
  constexpr int T = ChunkT<R>::value;
  constexpr int NG = T / TT;  // frequency groups per chunk
  static_assert(TT * sizeof(cplx<R>) == 16, "one 16-byte vector per (group, cell)");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Ks = reinterpret_cast<cplx<R>*>(smem_raw);  // [343][T]
  int4* Fs = reinterpret_cast<int4*>(Ks + kNOff * T);   // [NG][8][NQ] 16-byte vectors
  const HadTile tl = tiles[blockIdx.x];
  const int chunk = blockIdx.y;
  const int nthreads = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;

  // kernel spectra chunk (32 bytes per offset)
  {
    const int4* ksrc = reinterpret_cast<const int4*>(kspec + (size_t)tl.level * kstride + (size_t)chunk * kNOff * T);
    int4* kdst = reinterpret_cast<int4*>(Ks);
    const int4 zero4 = make_int4(0, 0, 0, 0);
    for (int i = tid; i < kNOff * 2; i += nthreads) {
      const int d = i >> 1;
      const int d0 = d / 49 - 3, d1 = (d / 7) % 7 - 3, d2 = d % 7 - 3;
      const bool near = d0 >= -1 && d0 <= 1 && d1 >= -1 && d1 <= 1 && d2 >= -1 && d2 <= 1;
      kdst[i] = (tl.excl_near && near) ? zero4 : ksrc[i];
    }
  }
  // source region chunk, natural cell order in HBM -> parity-major in shared memory
  const int R1 = tl.Rg[1], R2 = tl.Rg[2];
  const int NQ = tl.Rg[0] * R1 * R2;
  const int C1 = 2 * R1, C2 = 2 * R2;
  {
    const int4* fsrc = reinterpret_cast<const int4*>(spec + (size_t)chunk * spec_blocks * T);
    const int4 zero4 = make_int4(0, 0, 0, 0);
    for (int i = tid; i < 8 * NQ * NG; i += nthreads) {
      const int cell = i / NG, g = i % NG;
      const int x = cell / (C1 * C2), y = (cell / C2) % C1, z = cell % C2;
      const int b = ((x & 1) << 2) | ((y & 1) << 1) | (z & 1);
      const int q = ((x >> 1) * R1 + (y >> 1)) * R2 + (z >> 1);
      const int sid = src_ids[tl.src_off + cell];
      Fs[(g * 8 + b) * NQ + q] = sid >= 0 ? fsrc[(size_t)sid * NG + g] : zero4;
    }
  }
  __syncthreads();

  const int np = tl.P[0] * tl.P[1] * tl.P[2];
  const int pl = threadIdx.x;
  if (pl >= np) return;
  const int g = threadIdx.y;
  const int f0 = g * TT;
  const int pq[3] = {pl / (tl.P[1] * tl.P[2]), (pl / tl.P[2]) % tl.P[1], pl % tl.P[2]};
  // parent position inside the region
  const int q0 = tl.p0[0] + pq[0] - tl.r0[0], q1 = tl.p0[1] + pq[1] - tl.r0[1], q2 = tl.p0[2] + pq[2] - tl.r0[2];
  const cplx<R>* Fg = reinterpret_cast<const cplx<R>*>(Fs + (size_t)g * 8 * NQ);

  R ar[8][TT], ai[8][TT];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int t = 0; t < TT; ++t) { ar[a][t] = R(0); ai[a][t] = R(0); }

  for (int e = 0; e < 27; ++e) {
    const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
    if (tl.excl_near && e == 13) continue;
    const int n0 = q0 + e0, n1 = q1 + e1, n2 = q2 + e2;
    if (n0 < 0 || n0 >= tl.Rg[0] || n1 < 0 || n1 >= R1 || n2 < 0 || n2 >= R2) continue;
    const cplx<R>* fb = Fg + (size_t)((n0 * R1 + n1) * R2 + n2) * TT;
    // offset index of d = a - b - 2e is kbase + (a0-b0)*49 + (a1-b1)*7 + (a2-b2)
    const cplx<R>* kb = Ks + (size_t)off_index(-2 * e0, -2 * e1, -2 * e2) * T + f0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int b0 = b >> 2, b1 = (b >> 1) & 1, b2 = b & 1;
      R fr[TT], fi[TT];
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const cplx<R> v = fb[(size_t)b * NQ * TT + t];
        fr[t] = v.re; fi[t] = v.im;
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int a0 = a >> 2, a1 = (a >> 1) & 1, a2 = a & 1;
        const int dk = (a0 - b0) * 49 + (a1 - b1) * 7 + (a2 - b2);
#pragma unroll
        for (int t = 0; t < TT; ++t) {
          const cplx<R> k = kb[dk * T + t];
          ar[a][t] = fma(k.re, fr[t], ar[a][t]);
          ar[a][t] = fma(-k.im, fi[t], ar[a][t]);
          ai[a][t] = fma(k.re, fi[t], ai[a][t]);
          ai[a][t] = fma(k.im, fr[t], ai[a][t]);
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
    cplx<R>* o = acc + ((size_t)chunk * spec_blocks + sid) * T + f0;
#pragma unroll
    for (int t = 0; t < TT; ++t) o[t] = cplx<R>{ar[a][t], ai[a][t]};
  }
}

template <typename R>
cudaError_t launch_hadamard(int N, const HadTile* tiles, int ntiles, int max_parents, int max_region_cells,
                            const int* src_ids, const int* tgt_ids, const void* spec, void* acc, int spec_blocks,
                            const void* kspec, size_t kspec_level_stride, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  constexpr int T = ChunkT<R>::value;
  constexpr int TT = (sizeof(R) == 4) ? 2 : 1;
  const int ng = T / TT;
  int bx = ((max_parents + 31) / 32) * 32;
  if (bx * ng > 256) return cudaErrorInvalidConfiguration;
  const size_t sm = sizeof(cplx<R>) * T * ((size_t)kNOff + max_region_cells);
  if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(hadamard_kernel<R, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid(ntiles, nchunks<R>(N));
  dim3 block(bx, ng);
  hadamard_kernel<R, TT><<<grid, block, sm, s>>>(tiles, src_ids, tgt_ids, reinterpret_cast<const cplx<R>*>(spec),
                                                 reinterpret_cast<cplx<R>*>(acc), spec_blocks,
                                                 reinterpret_cast<const cplx<R>*>(kspec), kspec_level_stride);
  return cudaGetLastError();
}

template cudaError_t launch_hadamard<float>(int, const HadTile*, int, int, int, const int*, const int*, const void*,
                                            void*, int, const void*, size_t, cudaStream_t);
template cudaError_t launch_hadamard<double>(int, const HadTile*, int, int, int, const int*, const int*, const void*,
                                             void*, int, const void*, size_t, cudaStream_t);

}  // namespace flgf
