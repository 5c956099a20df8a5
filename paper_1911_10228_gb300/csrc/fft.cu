// a2 / a4: zero-padded (2N)^3 block FFTs for the block-wise convolution (Sec. 2.1).
//
// A source block holds N^3 values; the circular convolution of size 2N per
// axis with the (2N)^3 kernel array equals the linear one on the block
// (2N - 1 <= 2N points), so each block is zero-padded to (2N)^3, transformed
// with a real-to-complex FFT, multiplied with kernel spectra, and transformed
// back; only the first N^3 outputs are kept.
//
// Design (one CTA per block, whole 3-D transform in shared memory):
//   forward:  axis 2 (real, N nonzero of 2N) -> axis 1 -> axis 0, the last
//             pass written straight from registers into the chunked spectrum
//             layout in HBM.  Shared memory holds [N][2N][N+1] complex (the
//             axis-0 half that is nonzero before the last pass).
//   inverse:  axis 0 (only N outputs kept) -> axis 1 -> axis 2 (complex to
//             real, N outputs kept), reading the chunked spectrum layout.
// Each thread owns a whole line and transforms it in registers with a fully
// unrolled radix-2 FFT; the zero half of the input (forward) or the unused
// half of the output (inverse) is pruned by splitting the first (last)
// butterfly stage into two half-length transforms.
#include <cmath>

#include <type_traits>

#include "common.cuh"
#include "ffloat.cuh"
#include "internal.h"

namespace flgf {

// e^{-2 pi i j / 32}, j = 0..31, filled once from the host.
__constant__ double c_twd[32][2];
__constant__ float c_twf[32][2];
__constant__ float c_twff[32][4];  // (re hi, re lo, im hi, im lo)

cudaError_t fft_init_constants() {
  double td[32][2];
  float tf[32][2], tff[32][4];
  for (int j = 0; j < 32; ++j) {
    const long double a = -2.0L * 3.141592653589793238462643383279502884L * j / 32.0L;
    td[j][0] = (double)cosl(a);
    td[j][1] = (double)sinl(a);
    tf[j][0] = (float)td[j][0];
    tf[j][1] = (float)td[j][1];
    tff[j][0] = (float)cosl(a);
    tff[j][1] = (float)(cosl(a) - (long double)tff[j][0]);
    tff[j][2] = (float)sinl(a);
    tff[j][3] = (float)(sinl(a) - (long double)tff[j][2]);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_twd, td, sizeof(td));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_twff, tff, sizeof(tff));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_twf, tf, sizeof(tf));
}

template <typename R> __device__ __forceinline__ R tw_re(int j);
template <typename R> __device__ __forceinline__ R tw_im(int j);
template <> __device__ __forceinline__ double tw_re<double>(int j) { return c_twd[j][0]; }
template <> __device__ __forceinline__ double tw_im<double>(int j) { return c_twd[j][1]; }
template <> __device__ __forceinline__ float tw_re<float>(int j) { return c_twf[j][0]; }
template <> __device__ __forceinline__ float tw_im<float>(int j) { return c_twf[j][1]; }
template <> __device__ __forceinline__ ff tw_re<ff>(int j) { return ff(c_twff[j][0], c_twff[j][1]); }
template <> __device__ __forceinline__ ff tw_im<ff>(int j) { return ff(c_twff[j][2], c_twff[j][3]); }

// (tr, ti) = (wr + i wi)(xr + i xi).  Float-float takes each component as a
// two-term compensated dot product (DotAcc): one renormalisation instead of
// three.
template <typename R>
__device__ __forceinline__ void twiddle_mul(R wr, R wi, R xr, R xi, R& tr, R& ti) {
  if constexpr (std::is_same<R, ff>::value) {
    DotAcc<ff> a = DotAcc<ff>::prod(wr, xr);
    a.add(-wi, xi);
    DotAcc<ff> b = DotAcc<ff>::prod(wr, xi);
    b.add(wi, xr);
    tr = a.result();
    ti = b.result();
  } else {
    tr = wr * xr - wi * xi;
    ti = wr * xi + wi * xr;
  }
}

// In-register radix-2 FFT of length L (<= 32), natural order in and out.
// DIR = -1: forward (e^{-2 pi i jk/L}); DIR = +1: inverse without
// normalisation.  Recursive even/odd split: every array index is a
// compile-time constant, so the arrays live in registers.
template <int L, int DIR, typename R>
struct RegFFT {
  static __device__ __forceinline__ void run(R* re, R* im) {
    constexpr int H = L / 2;
    R er[H], ei[H], odr[H], odi[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      er[j] = re[2 * j]; ei[j] = im[2 * j];
      odr[j] = re[2 * j + 1]; odi[j] = im[2 * j + 1];
    }
    RegFFT<H, DIR, R>::run(er, ei);
    RegFFT<H, DIR, R>::run(odr, odi);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      R tr, ti;
      if (k == 0) {
        tr = odr[k]; ti = odi[k];
      } else if (4 * k == L) {  // w = -i (forward) or +i (inverse)
        tr = DIR < 0 ? odi[k] : -odi[k];
        ti = DIR < 0 ? -odr[k] : odr[k];
      } else {
        const R wr = tw_re<R>(k * (32 / L));
        const R wi = DIR < 0 ? tw_im<R>(k * (32 / L)) : -tw_im<R>(k * (32 / L));
        twiddle_mul(wr, wi, odr[k], odi[k], tr, ti);
      }
      re[k] = er[k] + tr; im[k] = ei[k] + ti;
      re[k + H] = er[k] - tr; im[k + H] = ei[k] - ti;
    }
  }
};
template <int DIR, typename R>
struct RegFFT<1, DIR, R> {
  static __device__ __forceinline__ void run(R*, R*) {}
};
template <int DIR, typename R>
struct RegFFT<2, DIR, R> {
  static __device__ __forceinline__ void run(R* re, R* im) {
    const R ar = re[0], ai = im[0];
    re[0] = ar + re[1]; im[0] = ai + im[1];
    re[1] = ar - re[1]; im[1] = ai - im[1];
  }
};

template <int L, int DIR, typename R>
__device__ __forceinline__ void fft_reg(R* re, R* im) {
  RegFFT<L, DIR, R>::run(re, im);
}

// Forward FFT of length L whose inputs L/2..L-1 are zero.  out(k, re, im) is
// called for every k = 0..L-1 (even k first).
template <int L, typename R, typename Out>
__device__ __forceinline__ void fft_fwd_pruned(const R* xr, const R* xi, Out out) {
  constexpr int H = L / 2;
  R ar[H], ai[H];
#pragma unroll
  for (int j = 0; j < H; ++j) { ar[j] = xr[j]; ai[j] = xi[j]; }
  fft_reg<H, -1>(ar, ai);
#pragma unroll
  for (int m = 0; m < H; ++m) out(2 * m, ar[m], ai[m]);
#pragma unroll
  for (int j = 0; j < H; ++j) {
    if (j == 0) { ar[j] = xr[j]; ai[j] = xi[j]; continue; }
    const R wr = tw_re<R>(j * (32 / L)), wi = tw_im<R>(j * (32 / L));
    ar[j] = xr[j] * wr - xi[j] * wi;
    ai[j] = xr[j] * wi + xi[j] * wr;
  }
  fft_reg<H, -1>(ar, ai);
#pragma unroll
  for (int m = 0; m < H; ++m) out(2 * m + 1, ar[m], ai[m]);
}

// Inverse FFT (no normalisation) of length L, only outputs 0..L/2-1.
template <int L, typename R>
__device__ __forceinline__ void fft_inv_pruned(const R* Xr, const R* Xi, R* xr, R* xi) {
  constexpr int H = L / 2;
  R er[H], ei[H], odr[H], odi[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    er[m] = Xr[2 * m]; ei[m] = Xi[2 * m];
    odr[m] = Xr[2 * m + 1]; odi[m] = Xi[2 * m + 1];
  }
  fft_reg<H, +1>(er, ei);
  fft_reg<H, +1>(odr, odi);
#pragma unroll
  for (int j = 0; j < H; ++j) {
    if (j == 0) { xr[j] = er[j] + odr[j]; xi[j] = ei[j] + odi[j]; continue; }
    const R wr = tw_re<R>(j * (32 / L)), wi = -tw_im<R>(j * (32 / L));
    if constexpr (std::is_same<R, ff>::value) {
      R tr, ti;
      twiddle_mul(wr, wi, odr[j], odi[j], tr, ti);
      xr[j] = er[j] + tr;
      xi[j] = ei[j] + ti;
    } else {
      xr[j] = er[j] + (odr[j] * wr - odi[j] * wi);
      xi[j] = ei[j] + (odr[j] * wi + odi[j] * wr);
    }
  }
}

// ---------------------------------------------------------------------------
// Forward transform of source blocks.
// ---------------------------------------------------------------------------
// R: storage type of the block values and spectra; C: arithmetic type of the
// transform (R itself; the inverse also runs with the compensated ff on FP32
// data).
template <typename R, int N, typename C>
__global__ void __launch_bounds__(N * N) fft_fwd_kernel(const R* __restrict__ nodes, const int* __restrict__ gids,
                                                        const int* __restrict__ sids, cplx<R>* __restrict__ spec,
                                                        int spec_blocks) {
  constexpr int P = 2 * N, NX = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<C>* buf = reinterpret_cast<cplx<C>*>(smem_raw);  // [N z][P y][NX kx]
  const int gid = gids[blockIdx.x], sid = sids[blockIdx.x];
  const R* in = nodes + (size_t)gid * N * N * N;
  const int tid = threadIdx.x;

  // stage the block with coalesced 16-byte loads: plane z goes to the rows
  // y >= N of plane z of the buffer, which axis 2 leaves untouched.  Staged
  // rows are SU (odd) 16-byte vectors apart, so the 8 lanes of a quarter warp
  // reading 8 consecutive rows hit 8 different bank groups.
  constexpr int V = 16 / (int)sizeof(R);  // values per 16-byte vector
  constexpr int RV = N / V;               // vectors per row
  constexpr int SU = RV + 1;              // staged row stride in vectors
  static_assert(N * SU * 16 <= N * NX * (int)sizeof(cplx<C>), "staged plane fits the unused rows");
  {
    const int4* src = reinterpret_cast<const int4*>(in);
    for (int i = tid; i < N * N * RV; i += blockDim.x) {
      const int z = i / (N * RV), y = (i / RV) % N, u = i % RV;
      reinterpret_cast<int4*>(buf + (z * P + N) * NX)[y * SU + u] = __ldg(src + i);
    }
  }
  __syncthreads();
  // axis 2 (real input, N of 2N nonzero)
  for (int line = tid; line < N * N; line += blockDim.x) {
    const int z = line / N, y = line % N;
    C xr[N], xi[N];
    const int4* stage = reinterpret_cast<const int4*>(buf + (z * P + N) * NX) + y * SU;
#pragma unroll
    for (int u = 0; u < RV; ++u) {
      const int4 v = stage[u];
      const R* r = reinterpret_cast<const R*>(&v);
#pragma unroll
      for (int j = 0; j < V; ++j) { xr[u * V + j] = Arith<C>::from(r[j]); xi[u * V + j] = C(0.0f); }
    }
    cplx<C>* row = buf + (z * P + y) * NX;
    fft_fwd_pruned<P>(xr, xi, [&](int k, C re, C im) {
      if (k <= N) row[k] = cplx<C>{re, im};
    });
  }
  __syncthreads();
  // axis 1 (N of 2N nonzero)
  for (int line = tid; line < N * NX; line += blockDim.x) {
    const int z = line / NX, kx = line % NX;
    C xr[N], xi[N];
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const cplx<C> v = buf[(z * P + y) * NX + kx];
      xr[y] = v.re; xi[y] = v.im;
    }
    fft_fwd_pruned<P>(xr, xi, [&](int k, C re, C im) { buf[(z * P + k) * NX + kx] = cplx<C>{re, im}; });
  }
  __syncthreads();
  // axis 0 (N of 2N nonzero) -> HBM, chunked layout
  for (int line = tid; line < P * NX; line += blockDim.x) {
    const int ky = line / NX, kx = line % NX;
    C xr[N], xi[N];
#pragma unroll
    for (int z = 0; z < N; ++z) {
      const cplx<C> v = buf[(z * P + ky) * NX + kx];
      xr[z] = v.re; xi[z] = v.im;
    }
    fft_fwd_pruned<P>(xr, xi, [&](int k, C re, C im) {
      const int w = (k * P + ky) * NX + kx;
      spec[spec_index<R>(w, sid, spec_blocks)] = cplx<R>{Arith<C>::template to<R>(re), Arith<C>::template to<R>(im)};
    });
  }
}

// ---------------------------------------------------------------------------
// Inverse transform of accumulated spectra; keeps the first N^3 outputs.
// ---------------------------------------------------------------------------
// TH threads per block.  With N (N + 1) threads the 2N (N + 1) lines of the
// first axis take exactly two rounds and the N (N + 1) of the second one (N^2
// threads leave the last round of each nearly empty).
template <typename R, int N, typename C, int TH>
__global__ void __launch_bounds__(TH) fft_inv_kernel(const cplx<R>* __restrict__ acc, int spec_blocks,
                                                        const int* __restrict__ sids, const int* __restrict__ gids,
                                                        const double* __restrict__ scales, R* __restrict__ out) {
  constexpr int P = 2 * N, NX = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<C>* buf = reinterpret_cast<cplx<C>*>(smem_raw);  // [N z][P y][NX kx]
  const int sid = sids[blockIdx.x], gid = gids[blockIdx.x];
  const int tid = threadIdx.x;

  // axis 0: 2N inputs from HBM, keep z < N
  for (int line = tid; line < P * NX; line += blockDim.x) {
    const int ky = line / NX, kx = line % NX;
    C Xr[P], Xi[P];
#pragma unroll
    for (int kz = 0; kz < P; ++kz) {
      const cplx<R> v = acc[spec_index<R>((kz * P + ky) * NX + kx, sid, spec_blocks)];
      Xr[kz] = Arith<C>::from(v.re); Xi[kz] = Arith<C>::from(v.im);
    }
    C xr[N], xi[N];
    fft_inv_pruned<P>(Xr, Xi, xr, xi);
#pragma unroll
    for (int z = 0; z < N; ++z) buf[(z * P + ky) * NX + kx] = cplx<C>{xr[z], xi[z]};
  }
  __syncthreads();
  // axis 1: keep y < N
  for (int line = tid; line < N * NX; line += blockDim.x) {
    const int z = line / NX, kx = line % NX;
    C Xr[P], Xi[P];
#pragma unroll
    for (int ky = 0; ky < P; ++ky) {
      const cplx<C> v = buf[(z * P + ky) * NX + kx];
      Xr[ky] = v.re; Xi[ky] = v.im;
    }
    C xr[N], xi[N];
    fft_inv_pruned<P>(Xr, Xi, xr, xi);
#pragma unroll
    for (int y = 0; y < N; ++y) buf[(z * P + y) * NX + kx] = cplx<C>{xr[y], xi[y]};
  }
  __syncthreads();
  // axis 2: Hermitian half -> real, keep x < N
  const C scale = Arith<C>::from_d(scales[blockIdx.x] / (double)(P * P * P));
  R* o = out + (size_t)gid * N * N * N;
  for (int line = tid; line < N * N; line += blockDim.x) {
    const int z = line / N, y = line % N;
    const cplx<C>* row = buf + (z * P + y) * NX;
    C Xr[P], Xi[P];
#pragma unroll
    for (int k = 0; k <= N; ++k) { const cplx<C> v = row[k]; Xr[k] = v.re; Xi[k] = v.im; }
#pragma unroll
    for (int k = N + 1; k < P; ++k) { Xr[k] = Xr[P - k]; Xi[k] = -Xi[P - k]; }
    C xr[N], xi[N];
    fft_inv_pruned<P>(Xr, Xi, xr, xi);
    constexpr int V = 16 / (int)sizeof(R);
    int4* orow = reinterpret_cast<int4*>(o + (z * N + y) * N);
#pragma unroll
    for (int u = 0; u < N / V; ++u) {
      int4 v;
      R* r = reinterpret_cast<R*>(&v);
#pragma unroll
      for (int j = 0; j < V; ++j) r[j] = Arith<C>::template to<R>(scale * xr[u * V + j]);
      orow[u] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Inverse transform with two threads per line (float-float, N = 16).  The
// pruned 32-point inverse is x[n] = E[n] + w^n O[n] (n < 16) with E and O the
// 16-point inverses of the even and odd inputs: the even lane of a pair
// computes E, the odd lane O and w^n O, and the pair swaps halves with
// shuffles (the even lane keeps n < 8, the odd one n >= 8).  Half the
// registers of one thread per line, so 16 warps run without spilling
// (the arithmetic is the same as one thread per line, bit for bit).
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void half_line_inverse(int par, C (&hr)[16], C (&hi)[16], C (&xr)[8], C (&xi)[8]) {
  constexpr int H = 16;
  fft_reg<H, +1>(hr, hi);
  if (par) {
#pragma unroll
    for (int j = 1; j < H; ++j) {
      C tr, ti;
      twiddle_mul(tw_re<C>(j), -tw_im<C>(j), hr[j], hi[j], tr, ti);
      hr[j] = tr;
      hi[j] = ti;
    }
  }
  // even lane sends E[8 + i], odd lane sends (w O)[i]
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const C sr = par ? hr[i] : hr[8 + i], si = par ? hi[i] : hi[8 + i];
    C rr, ri;
    rr.hi = __shfl_xor_sync(0xffffffffu, sr.hi, 1);
    rr.lo = __shfl_xor_sync(0xffffffffu, sr.lo, 1);
    ri.hi = __shfl_xor_sync(0xffffffffu, si.hi, 1);
    ri.lo = __shfl_xor_sync(0xffffffffu, si.lo, 1);
    // even: x[i] = E[i] + (w O)[i]; odd: x[8 + i] = E[8 + i] + (w O)[8 + i]
    xr[i] = par ? rr + hr[8 + i] : hr[i] + rr;
    xi[i] = par ? ri + hi[8 + i] : hi[i] + ri;
  }
}

template <typename R, int N, typename C, int TH>
__global__ void __launch_bounds__(TH) fft_inv2_kernel(const cplx<R>* __restrict__ acc, int spec_blocks,
                                                     const int* __restrict__ sids, const int* __restrict__ gids,
                                                     const double* __restrict__ scales, R* __restrict__ out) {
  constexpr int P = 2 * N, NX = N + 1, HL = N / 2;
  static_assert(N == 16, "two threads per line: N = 16");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<C>* buf = reinterpret_cast<cplx<C>*>(smem_raw);  // [N z][P y][NX kx]
  const int sid = sids[blockIdx.x], gid = gids[blockIdx.x];
  const int par = threadIdx.x & 1, pt = threadIdx.x >> 1;
  constexpr int PAIRS = TH / 2;
  // axis 0: 2N inputs from HBM (this lane: kz = 2 m + par), keep z < N
  for (int l0 = 0; l0 < P * NX; l0 += PAIRS) {
    const int line = l0 + pt;
    const bool on = line < P * NX;  // pairs past the end idle (uniform per pair)
    const int ky = on ? line / NX : 0, kx = on ? line % NX : 0;
    C hr[16], hi[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const cplx<R> v = acc[spec_index<R>(((2 * m + par) * P + ky) * NX + kx, sid, spec_blocks)];
      hr[m] = Arith<C>::from(v.re); hi[m] = Arith<C>::from(v.im);
    }
    C xr[8], xi[8];
    half_line_inverse<C>(par, hr, hi, xr, xi);
    if (on) {
#pragma unroll
      for (int i = 0; i < HL; ++i) buf[((par * HL + i) * P + ky) * NX + kx] = cplx<C>{xr[i], xi[i]};
    }
  }
  __syncthreads();
  // axis 1: keep y < N
  for (int l0 = 0; l0 < N * NX; l0 += PAIRS) {
    const int line = l0 + pt;
    const bool on = line < N * NX;
    const int z = on ? line / NX : 0, kx = on ? line % NX : 0;
    C hr[16], hi[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const cplx<C> v = buf[(z * P + 2 * m + par) * NX + kx];
      hr[m] = v.re; hi[m] = v.im;
    }
    C xr[8], xi[8];
    half_line_inverse<C>(par, hr, hi, xr, xi);
    __syncwarp();
    if (on) {
#pragma unroll
      for (int i = 0; i < HL; ++i) buf[(z * P + par * HL + i) * NX + kx] = cplx<C>{xr[i], xi[i]};
    }
  }
  __syncthreads();
  // axis 2: Hermitian half -> real, keep x < N
  const C scale = Arith<C>::from_d(scales[blockIdx.x] / (double)(P * P * P));
  R* o = out + (size_t)gid * N * N * N;
  for (int l0 = 0; l0 < N * N; l0 += PAIRS) {
    const int line = l0 + pt;
    const bool on = line < N * N;
    const int z = on ? line / N : 0, y = on ? line % N : 0;
    const cplx<C>* row = buf + (z * P + y) * NX;
    C hr[16], hi[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int k = 2 * m + par;  // X[k] for k > N is conj(X[P - k])
      const cplx<C> v = row[k <= N ? k : P - k];
      hr[m] = v.re; hi[m] = k <= N ? v.im : -v.im;
    }
    C xr[8], xi[8];
    half_line_inverse<C>(par, hr, hi, xr, xi);
    if (on) {
      float4 q[2];
      float* r = reinterpret_cast<float*>(q);
#pragma unroll
      for (int i = 0; i < HL; ++i) r[i] = Arith<C>::template to<R>(scale * xr[i]);
      float4* orow = reinterpret_cast<float4*>(o + (z * N + y) * N + par * HL);
      orow[0] = q[0];
      orow[1] = q[1];
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel spectra (setup, FP64): full 2N along axes 2 and 1, the 2N axis-0
// planes split into two halves of N that are transformed as pruned inputs
// and combined as LO + (-1)^{k0} HI.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(N * N) fft_kernel_half(const double* __restrict__ karr, int zoff,
                                                         cplx<double>* __restrict__ out) {
  constexpr int P = 2 * N, NX = N + 1, NW = P * P * NX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem_raw);  // [N z][P y][NX kx]
  const int d = blockIdx.x;
  const double* in = karr + (size_t)d * P * P * P;
  const int tid = threadIdx.x;
  for (int line = tid; line < N * P; line += blockDim.x) {
    const int z = line / P, y = line % P;
    double xr[P], xi[P];
#pragma unroll
    for (int x = 0; x < P; ++x) { xr[x] = in[((z + zoff) * P + y) * P + x]; xi[x] = 0.0; }
    fft_reg<P, -1>(xr, xi);
#pragma unroll
    for (int k = 0; k <= N; ++k) buf[(z * P + y) * NX + k] = cplx<double>{xr[k], xi[k]};
  }
  __syncthreads();
  for (int line = tid; line < N * NX; line += blockDim.x) {
    const int z = line / NX, kx = line % NX;
    double xr[P], xi[P];
#pragma unroll
    for (int y = 0; y < P; ++y) { const cplx<double> v = buf[(z * P + y) * NX + kx]; xr[y] = v.re; xi[y] = v.im; }
    fft_reg<P, -1>(xr, xi);
#pragma unroll
    for (int y = 0; y < P; ++y) buf[(z * P + y) * NX + kx] = cplx<double>{xr[y], xi[y]};
  }
  __syncthreads();
  cplx<double>* o = out + (size_t)d * NW;
  for (int line = tid; line < P * NX; line += blockDim.x) {
    const int ky = line / NX, kx = line % NX;
    double xr[N], xi[N];
#pragma unroll
    for (int z = 0; z < N; ++z) { const cplx<double> v = buf[(z * P + ky) * NX + kx]; xr[z] = v.re; xi[z] = v.im; }
    fft_fwd_pruned<P>(xr, xi, [&](int k, double re, double im) { o[(k * P + ky) * NX + kx] = cplx<double>{re, im}; });
  }
}

// Octree levels >= 1 never use the near offsets |d|_inf <= 1 (the near field
// belongs to the finest level), so their spectra are stored as zero.
template <typename R>
__global__ void kernel_combine(const cplx<double>* __restrict__ lo, const cplx<double>* __restrict__ hi, int N,
                               int zero_near, cplx<R>* __restrict__ kspec) {
  const int P = 2 * N, NX = N + 1, NW = P * P * NX;
  constexpr int T = ChunkT<R>::value;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)NW * kNOff) return;
  const int d = (int)(idx / NW), w = (int)(idx % NW);
  const int k0 = w / (P * NX);
  const cplx<double> a = lo[idx], b = hi[idx];
  const double sg = (k0 & 1) ? -1.0 : 1.0;
  const int dd0 = d / 49 - 3, dd1 = (d / 7) % 7 - 3, dd2 = d % 7 - 3;
  const bool near = dd0 >= -1 && dd0 <= 1 && dd1 >= -1 && dd1 <= 1 && dd2 >= -1 && dd2 <= 1;
  if (zero_near && near) {
    kspec[((size_t)(w / T) * kNOff + d) * T + (w % T)] = cplx<R>{R(0), R(0)};
    return;
  }
  // layout [chunk][343][T]
  kspec[((size_t)(w / T) * kNOff + d) * T + (w % T)] = cplx<R>{(R)(a.re + sg * b.re), (R)(a.im + sg * b.im)};
}

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R, typename C>
static cudaError_t launch_fwd(int N, const R* nodes, const int* gids, const int* sids, int count, cplx<R>* sp,
                              int spec_blocks, cudaStream_t s) {
  if (N == 16) {
    const size_t sm = sizeof(cplx<C>) * 16 * 32 * 17;
    cudaError_t e = set_smem(fft_fwd_kernel<R, 16, C>, sm);
    if (e != cudaSuccess) return e;
    fft_fwd_kernel<R, 16, C><<<count, 256, sm, s>>>(nodes, gids, sids, sp, spec_blocks);
  } else if (N == 8) {
    const size_t sm = sizeof(cplx<C>) * 8 * 16 * 9;
    fft_fwd_kernel<R, 8, C><<<count, 64, sm, s>>>(nodes, gids, sids, sp, spec_blocks);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Threads of the one-thread-per-line inverse kernel.  Transforms held in
// shared memory whole, one block per SM (FP64 at N = 16), take N (N + 1)
// threads: their arithmetic is the cost, and the first two axes then need no
// near-empty last round.  Plain FP32 keeps N^2 threads: it is bound by HBM,
// and at N (N + 1) threads its registers fit only two blocks per SM instead
// of three (measured on the 256^3 lattice: 0.19 ms at N^2, 0.25 ms at
// N (N + 1)).  Float-float at N = 16 runs the two-threads-per-line kernel
// with 512 threads (one-thread-per-line at 272 threads spilled; batched
// inverse FFTs 12.5 -> 10.9 ms).
template <typename C, int N> constexpr int inv_threads() {
  return std::is_same<C, float>::value ? N * N : N * (N + 1);
}
constexpr int kInv2Threads = 512;

template <typename R, typename C>
static cudaError_t launch_inv(int N, const cplx<R>* ac, int spec_blocks, const int* sids, const int* gids,
                              const double* scales, int count, R* out, cudaStream_t s) {
  if (N == 16) {
    const size_t sm = sizeof(cplx<C>) * 16 * 32 * 17;
    if constexpr (std::is_same<C, ff>::value) {
      constexpr int TH2 = kInv2Threads;
      cudaError_t e = set_smem(fft_inv2_kernel<R, 16, C, TH2>, sm);
      if (e != cudaSuccess) return e;
      fft_inv2_kernel<R, 16, C, TH2><<<count, TH2, sm, s>>>(ac, spec_blocks, sids, gids, scales, out);
    } else {
      constexpr int TH = inv_threads<C, 16>();
      cudaError_t e = set_smem(fft_inv_kernel<R, 16, C, TH>, sm);
      if (e != cudaSuccess) return e;
      fft_inv_kernel<R, 16, C, TH><<<count, TH, sm, s>>>(ac, spec_blocks, sids, gids, scales, out);
    }
  } else if (N == 8) {
    const size_t sm = sizeof(cplx<C>) * 8 * 16 * 9;
    constexpr int TH = inv_threads<C, 8>();
    fft_inv_kernel<R, 8, C, TH><<<count, TH, sm, s>>>(ac, spec_blocks, sids, gids, scales, out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_forward(int N, const R* nodes, const int* gids, const int* sids, int count, void* spec,
                               int spec_blocks, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  return launch_fwd<R, R>(N, nodes, gids, sids, count, reinterpret_cast<cplx<R>*>(spec), spec_blocks, s);
}

template <typename R>
cudaError_t launch_fft_inverse(int N, const void* acc, int spec_blocks, const int* sids, const int* gids,
                               const double* scales, int count, R* out, cudaStream_t s, bool compensated) {
  if (count <= 0) return cudaSuccess;
  const cplx<R>* ac = reinterpret_cast<const cplx<R>*>(acc);
  if constexpr (sizeof(R) == 4) {
    if (compensated) return launch_inv<R, ff>(N, ac, spec_blocks, sids, gids, scales, count, out, s);
  }
  return launch_inv<R, R>(N, ac, spec_blocks, sids, gids, scales, count, out, s);
}

template <typename R>
cudaError_t launch_kernel_spectra(int N, const double* karr, void* kspec_level, double* tmp, int zero_near, cudaStream_t s) {
  const int P = 2 * N, NW = P * P * (N + 1);
  cplx<double>* lo = reinterpret_cast<cplx<double>*>(tmp);
  cplx<double>* hi = lo + (size_t)kNOff * NW;
  const size_t sm = sizeof(cplx<double>) * N * P * (N + 1);
  cudaError_t e;
  if (N == 16) {
    if ((e = set_smem(fft_kernel_half<16>, sm)) != cudaSuccess) return e;
    fft_kernel_half<16><<<kNOff, 256, sm, s>>>(karr, 0, lo);
    fft_kernel_half<16><<<kNOff, 256, sm, s>>>(karr, 16, hi);
  } else if (N == 8) {
    fft_kernel_half<8><<<kNOff, 64, sm, s>>>(karr, 0, lo);
    fft_kernel_half<8><<<kNOff, 64, sm, s>>>(karr, 8, hi);
  } else {
    return cudaErrorInvalidValue;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t total = (size_t)NW * kNOff;
  kernel_combine<R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(lo, hi, N, zero_near,
                                                                     reinterpret_cast<cplx<R>*>(kspec_level));
  return cudaGetLastError();
}

template cudaError_t launch_fft_forward<float>(int, const float*, const int*, const int*, int, void*, int, cudaStream_t);
template cudaError_t launch_fft_forward<double>(int, const double*, const int*, const int*, int, void*, int,
                                                cudaStream_t);
template cudaError_t launch_fft_inverse<float>(int, const void*, int, const int*, const int*, const double*, int, float*,
                                               cudaStream_t, bool);
template cudaError_t launch_fft_inverse<double>(int, const void*, int, const int*, const int*, const double*, int,
                                                double*, cudaStream_t, bool);
template cudaError_t launch_kernel_spectra<float>(int, const double*, void*, double*, int, cudaStream_t);
template cudaError_t launch_kernel_spectra<double>(int, const double*, void*, double*, int, cudaStream_t);

}  // namespace flgf
