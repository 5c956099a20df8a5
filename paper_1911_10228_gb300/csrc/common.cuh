// Shared device-side definitions of the FLGF library (sm_103a).
//
// Spectrum layout ("chunked, frequency-major"): the R2C spectrum of a
// zero-padded (2N)^3 block has NW = 2N * 2N * (N+1) complex values; frequency
// w = (k0 * 2N + k1) * (N+1) + k2 (k2 is the Hermitian-halved axis, the last
// and fastest axis of the block's C-order data).  A chunk is T = 32 bytes /
// sizeof(complex) consecutive frequencies (4 complex floats or 2 complex
// doubles, one 32-byte sector), chunk = w / T.  Spectra of many blocks are
// stored as [chunk / 4][block][chunk % 4][T]: one block's four consecutive
// chunks form one 128-byte line.  The spectrum multiply-accumulate kernel
// reads and writes one sector per (chunk, block); the FFT kernels, whose
// consecutive lanes handle consecutive frequencies of one block, touch two
// whole 128-byte lines per warp-wide 8-byte access.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace flgf {

template <typename R> struct cplx { R re, im; };

template <typename R> struct ChunkT { static constexpr int value = 32 / (2 * (int)sizeof(R)); };

__host__ __device__ constexpr int nfreq(int N) { return 2 * N * 2 * N * (N + 1); }
template <typename R>
__host__ __device__ constexpr int nchunks(int N) { return nfreq(N) / ChunkT<R>::value; }

constexpr int kChunkGroup = 4;  // chunks per 128-byte line of one block

// Offset (in complex values) of chunk `chunk` of `block` in a spectrum array
// of `nblocks` blocks.
template <typename R>
__host__ __device__ __forceinline__ size_t chunk_offset(int chunk, int block, int nblocks) {
  constexpr int T = ChunkT<R>::value;
  return (((size_t)(chunk / kChunkGroup) * (size_t)nblocks + (size_t)block) * kChunkGroup + chunk % kChunkGroup) * T;
}

// Index of complex value (w, block) in a chunked spectrum array.
template <typename R>
__device__ __forceinline__ size_t spec_index(int w, int block, int nblocks) {
  constexpr int T = ChunkT<R>::value;
  return chunk_offset<R>(w / T, block, nblocks) + w % T;
}

// Number of relative block offsets d in [-3, 3]^3 whose kernel spectra are cached.
constexpr int kNOff = 343;
__host__ __device__ constexpr int off_index(int d0, int d1, int d2) {
  return ((d0 + 3) * 7 + (d1 + 3)) * 7 + (d2 + 3);
}

}  // namespace flgf
