// Small per-block operators around the convolution.
//
//  a1  anterpolation (upward pass, Sec. 2.1):  f~_P += sum_children (R_c0 x R_c1 x R_c2) f~_C,
//      R = J^T, J_c the N x N rows of the 1-D Lagrange matrix J_1 (2N x N) for child position c.
//  a5  interpolation (downward pass):           u~_C += (J_c0 x J_c1 x J_c2) u~_P.
//  a6  coarsening C (Sec. 3):                    coarse cell = mean of its 8 fine cells.
//  a8  coarse-fine interpolation J^l (Sec. 3):   quadratic, cell-centred, weights
//      (5/32, 15/16, -3/32) / mirrored, tensor product over a 3x3x3 coarse stencil.
//  a9  source correction:                        f^{l+1} -= L_Q^{(h_{l+1})} (J^l u~^l).
//  a10 7-point Laplacian L_Q^{(h)} u = (sum of 6 neighbours - 6 u) / h^2.
// All tensor-product operators are applied axis by axis in shared memory.
#include <cooperative_groups.h>

#include "common.cuh"
#include "ffloat.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace flgf {

// First parent node of the n_I-point Lagrange window of child node j
// (0..2N-1) for cell-centred nodes (child j at j + 1/2, parent p at 2p + 1, in
// child spacings): centred on the point, moved inwards at the faces.
template <int N, int NI>
__host__ __device__ constexpr int band_start(int j) {
  const int lo = j == 0 ? -1 : (j - 1) / 2;      // parent node just left of the point
  const int near = (j % 2 == 0) ? j / 2 : (j - 1) / 2;  // nearest parent node
  const int s = (NI % 2 == 0) ? lo - (NI / 2 - 1) : near - NI / 2;
  return s < 0 ? 0 : (s > N - NI ? N - NI : s);
}

// Shared-memory block with padded rows: element (i, j, k) at (i*N + j)*(N+1) + k.
template <int N>
__device__ __forceinline__ int pidx(int i, int j, int k) { return (i * N + j) * (N + 1) + k; }

// Position of child node j in its Lagrange window, in parent spacings from
// the window's first node: child nodes at j + 1/2, parent nodes at 2p + 1
// (child spacings), so t = (j + 1/2 - (2 s + 1)) / 2.
template <int N, int NI>
__host__ __device__ constexpr double window_pos(int j) {
  return (j - 2 * band_start<N, NI>(j) - 0.5) / 2.0;
}
// Newton coefficient of order k at t: forward t (t-1) ... (t-k+1) / k!
// (BACK = false) or backward t (t+1) ... (t+k-1) / k! (BACK = true).
template <bool BACK>
__host__ __device__ constexpr double newton_coef(double t, int k) {
  double c = 1.0;
  for (int i = 0; i < k; ++i) c *= (BACK ? t + i : t - i) / (i + 1);
  return c;
}

// One 1-D pass of interpolation (child position C along the axis) on a line
// held in registers: out[r] = the n_I-point Lagrange polynomial through the
// window's parent values, at child node C N + r.  Rows whose point lies in the
// central interval of their window use the Lagrange weights W (|w|_1 <= 1.3).
// The off-centre rows near the block faces, whose Lagrange weights alternate
// in sign with |w|_1 up to 7.2 (n_I = 6) and so would turn FP32 rounding into
// several ulps of error, evaluate the same polynomial in Newton form from the
// nearer end of the window: forward differences from its first node (point
// left of centre) or backward differences from its last node (right of
// centre), whose coefficients |c_k| stay small because the point is close to
// that end; for a smooth field the differences shrink with their order, so
// the rounding stays relative to the field value.
template <typename R, int N, int NI, int C>
__device__ __forceinline__ void line_interp(const R* in, R* out, const R* W) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int j = C * N + r;
    const int s = band_start<N, NI>(j);
    const double t = window_pos<N, NI>(j);
    const double mid = 0.5 * (NI - 1);
    if (t >= mid - 0.5 && t <= mid + 0.5) {
      DotAcc<R> acc = DotAcc<R>::zero();
#pragma unroll
      for (int m = 0; m < NI; ++m) acc.add(W[j * NI + m], in[s + m]);
      out[r] = acc.result();
    } else if (t < mid) {
      R d[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) d[i] = in[s + i];
#pragma unroll
      for (int k = 1; k < NI; ++k)
#pragma unroll
        for (int i = NI - 1; i >= k; --i) d[i] = d[i] - d[i - 1];  // d[k] = forward difference of order k at s
      DotAcc<R> acc = DotAcc<R>::prod(d[NI - 1], Arith<R>::from_d(newton_coef<false>(t, NI - 1)));
#pragma unroll
      for (int k = NI - 2; k >= 0; --k) acc.add(Arith<R>::from_d(newton_coef<false>(t, k)), d[k]);
      out[r] = acc.result();
    } else {
      R d[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) d[i] = in[s + NI - 1 - i];
#pragma unroll
      for (int k = 1; k < NI; ++k)
#pragma unroll
        for (int i = NI - 1; i >= k; --i) d[i] = d[i - 1] - d[i];  // d[k] = backward difference of order k at s + NI - 1
      const double tau = t - (NI - 1);
      DotAcc<R> acc = DotAcc<R>::prod(d[NI - 1], Arith<R>::from_d(newton_coef<true>(tau, NI - 1)));
#pragma unroll
      for (int k = NI - 2; k >= 0; --k) acc.add(Arith<R>::from_d(newton_coef<true>(tau, k)), d[k]);
      out[r] = acc.result();
    }
  }
}
// Its adjoint (anterpolation): out[q] += sum_r J[C N + r][q] in[r].
template <typename R, int N, int NI, int C>
__device__ __forceinline__ void line_anterp(const R* in, R* out, const R* W) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int j = C * N + r;
#pragma unroll
    for (int m = 0; m < NI; ++m) {
      const int q = band_start<N, NI>(j) + m;
      out[q] = fma(W[j * NI + m], in[r], out[q]);
    }
  }
}

// Load the banded weights W[j][m] = J1[j][band_start(j) + m] into shared memory.
template <typename R, int N, int NI>
__device__ __forceinline__ void load_band(const double* __restrict__ J1, R* W) {
  for (int i = threadIdx.x; i < 2 * N * NI; i += blockDim.x) {
    const int j = i / NI, m = i % NI;
    int s = (NI % 2 == 0) ? (j == 0 ? -1 : (j - 1) / 2) - (NI / 2 - 1) : ((j % 2 == 0) ? j / 2 : (j - 1) / 2) - NI / 2;
    s = s < 0 ? 0 : (s > N - NI ? N - NI : s);
    W[i] = Arith<R>::from_d(J1[j * N + s + m]);
  }
}

// a1: parent = sum over existing children of (R_c0 x R_c1 x R_c2) child.
// A cluster of 8 CTAs per parent, CTA rank c = child position (c0 c1 c2): each
// CTA applies the three 1-D passes to its own child (one thread per line, N^2
// threads; axis-2 lines are contiguous, padded rows keep the strided axis-1
// and axis-0 lines conflict-free) and leaves the result in its shared memory;
// after a cluster barrier CTA c sums slice c of the parent over the 8 CTAs'
// shared memory (distributed shared memory, fixed order) and writes it.  The
// 8 children of a parent are thus transformed at the same time, not one
// after another, and nothing but the parent goes back to HBM.
template <typename R, int N, int NI>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(N * N)
    anterp_kernel(const double* __restrict__ J1, const int* __restrict__ parents, const int* __restrict__ children,
                  R* __restrict__ nodes) {
  constexpr int N3 = N * N * N, PS = N * N * (N + 1);
  constexpr int V = 16 / (int)sizeof(R);  // values per 16-byte vector
  constexpr int PER = N3 / V / (N * N);    // vectors per thread
  static_assert(N % V == 0 && PER * V * N * N == N3, "whole vectors per thread");
  __shared__ R W[2 * N * NI];
  __shared__ __align__(16) R A[PS];
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int pi = blockIdx.x / 8;
  load_band<R, N, NI>(J1, W);
  const int t = threadIdx.x, u = t / N, v = t % N;
  const int cid = children[pi * 8 + c];
  R acc[N];
#pragma unroll
  for (int q = 0; q < N; ++q) acc[q] = R(0);
  if (cid >= 0) {
    const int c0 = c >> 2, c1 = (c >> 1) & 1, c2 = c & 1;
    const int4* src = reinterpret_cast<const int4*>(nodes + (size_t)cid * N3);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int4 val = __ldg(src + t + p * N * N);
      const int i = (t + p * N * N) * V;  // V consecutive values of one row
      const R* pv = reinterpret_cast<const R*>(&val);
#pragma unroll
      for (int j = 0; j < V; ++j) A[pidx<N>(i / (N * N), (i / N) % N, i % N + j)] = pv[j];
    }
    __syncthreads();
    R in[N], out[N];
    // axis 2: line (u, v) = A[u][v][:]
#pragma unroll
    for (int k = 0; k < N; ++k) { in[k] = A[pidx<N>(u, v, k)]; out[k] = R(0); }
    if (c2) line_anterp<R, N, NI, 1>(in, out, W); else line_anterp<R, N, NI, 0>(in, out, W);
#pragma unroll
    for (int k = 0; k < N; ++k) A[pidx<N>(u, v, k)] = out[k];
    __syncthreads();
    // axis 1: line (u, v) = A[u][:][v]
#pragma unroll
    for (int j = 0; j < N; ++j) { in[j] = A[pidx<N>(u, j, v)]; out[j] = R(0); }
    if (c1) line_anterp<R, N, NI, 1>(in, out, W); else line_anterp<R, N, NI, 0>(in, out, W);
#pragma unroll
    for (int j = 0; j < N; ++j) A[pidx<N>(u, j, v)] = out[j];
    __syncthreads();
    // axis 0: line (u, v) = A[:][u][v]
#pragma unroll
    for (int i = 0; i < N; ++i) in[i] = A[pidx<N>(i, u, v)];
    if (c0) line_anterp<R, N, NI, 1>(in, acc, W); else line_anterp<R, N, NI, 0>(in, acc, W);
    __syncthreads();
  }
  // this child's contribution, dense [i][u][v] (an absent child contributes zero)
#pragma unroll
  for (int i = 0; i < N; ++i) A[(i * N + u) * N + v] = acc[i];
  cluster.sync();
  // slice c of the parent: sum over the 8 CTAs in rank order
  constexpr int SL = N3 / 8;
  R* dst = nodes + (size_t)parents[pi] * N3;
  for (int i = c * SL + t; i < (c + 1) * SL; i += N * N) {
    R sum = R(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += cluster.map_shared_rank(A, q)[i];
    dst[i] = sum;
  }
  cluster.sync();  // no CTA leaves while others still read its shared memory
}

// a1 for levels with many parents: one CTA per parent walks its existing
// children in rank order (the same three passes per child) and adds each
// child's contribution to its running sum in that order, so the parent is
// bit-identical to the cluster form's, without CTAs for absent children
// (sparse octrees have three children per parent on average).
template <typename R, int N, int NI>
__global__ void __launch_bounds__(N * N) anterp_seq_kernel(const double* __restrict__ J1, const int* __restrict__ parents,
                                                           const int* __restrict__ children, R* __restrict__ nodes) {
  constexpr int N3 = N * N * N, PS = N * N * (N + 1);
  constexpr int V = 16 / (int)sizeof(R);
  constexpr int PER = N3 / V / (N * N);
  __shared__ R W[2 * N * NI];
  __shared__ __align__(16) R A[PS];
  load_band<R, N, NI>(J1, W);
  const int t = threadIdx.x, u = t / N, v = t % N;
  const int pi = blockIdx.x;
  R tot[N];
#pragma unroll
  for (int q = 0; q < N; ++q) tot[q] = R(0);
  for (int c = 0; c < 8; ++c) {
    const int cid = children[pi * 8 + c];
    if (cid < 0) continue;  // uniform over the CTA
    const int c0 = c >> 2, c1 = (c >> 1) & 1, c2 = c & 1;
    const int4* src = reinterpret_cast<const int4*>(nodes + (size_t)cid * N3);
    __syncthreads();  // the previous child's last pass has read A
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int4 val = __ldg(src + t + p * N * N);
      const int i = (t + p * N * N) * V;
      const R* pv = reinterpret_cast<const R*>(&val);
#pragma unroll
      for (int j = 0; j < V; ++j) A[pidx<N>(i / (N * N), (i / N) % N, i % N + j)] = pv[j];
    }
    __syncthreads();
    R in[N], out[N];
#pragma unroll
    for (int k = 0; k < N; ++k) { in[k] = A[pidx<N>(u, v, k)]; out[k] = R(0); }
    if (c2) line_anterp<R, N, NI, 1>(in, out, W); else line_anterp<R, N, NI, 0>(in, out, W);
#pragma unroll
    for (int k = 0; k < N; ++k) A[pidx<N>(u, v, k)] = out[k];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N; ++j) { in[j] = A[pidx<N>(u, j, v)]; out[j] = R(0); }
    if (c1) line_anterp<R, N, NI, 1>(in, out, W); else line_anterp<R, N, NI, 0>(in, out, W);
#pragma unroll
    for (int j = 0; j < N; ++j) A[pidx<N>(u, j, v)] = out[j];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) { in[i] = A[pidx<N>(i, u, v)]; out[i] = R(0); }
    if (c0) line_anterp<R, N, NI, 1>(in, out, W); else line_anterp<R, N, NI, 0>(in, out, W);
#pragma unroll
    for (int i = 0; i < N; ++i) tot[i] += out[i];
  }
  R* dst = nodes + (size_t)parents[pi] * N3;
#pragma unroll
  for (int i = 0; i < N; ++i) dst[(i * N + u) * N + v] = tot[i];
}

// a5: child += (J_c0 x J_c1 x J_c2) parent, in arithmetic type C: R, or the
// compensated ff for FP32 data (the three passes then keep their intermediate
// lines in float-float, so the rounding of one pass is not amplified by the
// extrapolating rows of the next).
template <typename R, int N, int NI, typename C = R>
__global__ void __launch_bounds__(N * N) interp_add_kernel(const double* __restrict__ J1, const int* __restrict__ childs,
                                                           const int* __restrict__ parents, const int* __restrict__ cpos,
                                                           R* __restrict__ unodes) {
  constexpr int N3 = N * N * N, PS = N * N * (N + 1);
  __shared__ C W[2 * N * NI];
  __shared__ C A[PS];  // each thread transforms whole lines in place
  load_band<C, N, NI>(J1, W);
  const int t = threadIdx.x, u = t / N, v = t % N;
  const int c = cpos[blockIdx.x];
  const int c0 = c >> 2, c1 = (c >> 1) & 1, c2 = c & 1;
  const R* src = unodes + (size_t)parents[blockIdx.x] * N3;
  for (int i = t; i < N3; i += blockDim.x) A[pidx<N>(i / (N * N), (i / N) % N, i % N)] = Arith<C>::from(src[i]);
  __syncthreads();
  C in[N], out[N];
#pragma unroll
  for (int k = 0; k < N; ++k) in[k] = A[pidx<N>(u, v, k)];
  if (c2) line_interp<C, N, NI, 1>(in, out, W); else line_interp<C, N, NI, 0>(in, out, W);
#pragma unroll
  for (int k = 0; k < N; ++k) A[pidx<N>(u, v, k)] = out[k];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) in[j] = A[pidx<N>(u, j, v)];
  if (c1) line_interp<C, N, NI, 1>(in, out, W); else line_interp<C, N, NI, 0>(in, out, W);
#pragma unroll
  for (int j = 0; j < N; ++j) A[pidx<N>(u, j, v)] = out[j];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) in[i] = A[pidx<N>(i, u, v)];
  if (c0) line_interp<C, N, NI, 1>(in, out, W); else line_interp<C, N, NI, 0>(in, out, W);
  R* dst = unodes + (size_t)childs[blockIdx.x] * N3;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    R& d = dst[(i * N + u) * N + v];
    d = Arith<C>::template to<R>(Arith<C>::from(d) + out[i]);
  }
}

// Block copies (or zero fills) in 16-byte vectors: a block is N^3 values
// (a multiple of 16 bytes) at a 16-byte aligned offset of its array.
template <typename R>
__global__ void copy_blocks_kernel(int N, const R* __restrict__ src, const int* __restrict__ src_ids,
                                   R* __restrict__ dst, const int* __restrict__ dst_ids,
                                   const uint8_t* __restrict__ zero) {
  const int N3 = N * N * N;
  const int nv = N3 * (int)sizeof(R) / 16;
  const int i = blockIdx.x;
  const bool z = zero != nullptr && zero[i];
  int4* d = reinterpret_cast<int4*>(dst + (size_t)dst_ids[i] * N3);
  if (z) {
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d[e] = make_int4(0, 0, 0, 0);
  } else {
    const int4* s = reinterpret_cast<const int4*>(src + (size_t)src_ids[i] * N3);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) d[e] = __ldg(s + e);
  }
}

template <typename R>
__global__ void coarsen_kernel(int N, const R* __restrict__ fine_f, const int* __restrict__ fine_ids,
                               R* __restrict__ coarse_f, const int* __restrict__ coarse_ids) {
  const int N3 = N * N * N, H = N / 2;
  R* out = coarse_f + (size_t)coarse_ids[blockIdx.x] * N3;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int i = o / (N * N), j = (o / N) % N, k = o % N;
    const int a = ((i >= H) << 2) | ((j >= H) << 1) | (k >= H);
    const R* f = fine_f + (size_t)fine_ids[blockIdx.x * 8 + a] * N3;
    const int fi = 2 * (i % H), fj = 2 * (j % H), fk = 2 * (k % H);
    R s = 0;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) s += f[((fi + di) * N + fj + dj) * N + fk + dk];
    out[o] = s * R(0.125);
  }
}

// Quadratic cell-centred weights on coarse cells (i-1, i, i+1) for the fine
// cell at -1/4 (sub = 0) and +1/4 (sub = 1) of coarse cell i.
template <typename R>
__device__ __forceinline__ R cf_w(int sub, int e) {  // exact in FP32 and FP64
  const int i = sub == 0 ? e : 2 - e;
  return i == 0 ? R(5.0 / 32.0) : (i == 1 ? R(15.0 / 16.0) : R(-3.0 / 32.0));
}

template <typename R, int N, int MODE>
__global__ void __launch_bounds__(N >= 16 ? 256 : 128)
    cf_interp_kernel(const R* __restrict__ ucoarse, const int* __restrict__ nbr27, const int* __restrict__ fine_ids,
                     const int* __restrict__ cposv, R* __restrict__ fine, const double* __restrict__ inv_hf2,
                     int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int mode = MODE;
  constexpr int N3 = N * N * N;
  constexpr int halo = mode == 1 ? 1 : 0;
  constexpr int F = N + 2 * halo;          // fine region extent
  constexpr int M = N / 2 + 2 + 2 * halo;  // coarse region extent
  R* C = reinterpret_cast<R*>(smem_raw);  // [M][M][M]
  R* T1 = C + M * M * M;                  // [M][M][F]
  R* T2 = T1 + M * M * F;                 // [M][F][F]
  R* U = T2 + M * F * F;                  // [F][F][F]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c = cposv[blockIdx.x];
  const int cp[3] = {c >> 2, (c >> 1) & 1, c & 1};
  // fine region cell g (0..F-1) is fine index g - halo relative to the child
  // block, i.e. G = cp*N + g - halo relative to the parent block's fine origin;
  // its coarse cell is G >> 1.  Coarse region starts at cbase = ((cp*N - halo) >> 1) - 1.
  int cbase[3];
  for (int a = 0; a < 3; ++a) cbase[a] = ((cp[a] * N - halo) >> 1) - 1;
  const int* nb = nbr27 + (size_t)blockIdx.x * 27;
  for (int o = tid; o < M * M * M; o += nt) {
    const int x[3] = {o / (M * M) + cbase[0], (o / M) % M + cbase[1], o % M + cbase[2]};
    int e[3], loc[3];
    for (int a = 0; a < 3; ++a) {
      e[a] = x[a] < 0 ? -1 : (x[a] >= N ? 1 : 0);
      loc[a] = x[a] - e[a] * N;
    }
    const int b = nb[(e[0] + 1) * 9 + (e[1] + 1) * 3 + (e[2] + 1)];
    R v = 0;
    if (b >= 0) {
      v = ucoarse[(size_t)b * N3 + (loc[0] * N + loc[1]) * N + loc[2]];
    } else if (err_flag) {
      atomicExch(err_flag, 1);
    }
    C[o] = v;
  }
  __syncthreads();
  // axis 2: T1[i][j][g] = sum_e w(sub, e) C[i][j][ci + e - 1 - cbase]
  for (int o = tid; o < M * M * F; o += nt) {
    const int g = o % F, ij = o / F;
    const int G = cp[2] * N + g - halo, ci = (G >> 1) - cbase[2], sub = G & 1;
    R s = 0;
    for (int e = 0; e < 3; ++e) s += cf_w<R>(sub, e) * C[ij * M + ci + e - 1];
    T1[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < M * F * F; o += nt) {  // axis 1
    const int k = o % F, g = (o / F) % F, i = o / (F * F);
    const int G = cp[1] * N + g - halo, ci = (G >> 1) - cbase[1], sub = G & 1;
    R s = 0;
    for (int e = 0; e < 3; ++e) s += cf_w<R>(sub, e) * T1[(i * M + ci + e - 1) * F + k];
    T2[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < F * F * F; o += nt) {  // axis 0
    const int jk = o % (F * F), g = o / (F * F);
    const int G = cp[0] * N + g - halo, ci = (G >> 1) - cbase[0], sub = G & 1;
    R s = 0;
    for (int e = 0; e < 3; ++e) s += cf_w<R>(sub, e) * T2[(ci + e - 1) * F * F + jk];
    U[o] = s;
  }
  __syncthreads();
  R* dst = fine + (size_t)fine_ids[blockIdx.x] * N3;
  if (mode == 0) {
    for (int o = tid; o < N3; o += nt) dst[o] += U[o];
  } else {
    const R ih2 = (R)inv_hf2[blockIdx.x];
    for (int o = tid; o < N3; o += nt) {
      const int i = o / (N * N) + 1, j = (o / N) % N + 1, k = o % N + 1;
      const int q = (i * F + j) * F + k;
      const R lap = U[q + F * F] + U[q - F * F] + U[q + F] + U[q - F] + U[q + 1] + U[q - 1] - R(6) * U[q];
      dst[o] -= lap * ih2;
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint (transpose) operators for gradients.
// ---------------------------------------------------------------------------

// dst[dst_ids[i]] (+)= (s1_ids[i] >= 0 ? s1[s1_ids[i]] : 0) + (s2_ids[i] >= 0 ? s2[s2_ids[i]] : 0)
template <typename R>
__global__ void combine_blocks_kernel(int N, R* __restrict__ dst, const int* __restrict__ dst_ids,
                                      const R* __restrict__ s1, const int* __restrict__ s1_ids,
                                      const R* __restrict__ s2, const int* __restrict__ s2_ids, int accumulate) {
  const int N3 = N * N * N;
  const int i = blockIdx.x;
  const int a = s1_ids[i], b = s2_ids ? s2_ids[i] : -1;
  R* d = dst + (size_t)dst_ids[i] * N3;
  for (int e = threadIdx.x; e < N3; e += blockDim.x) {
    R v = R(0);
    if (a >= 0) v += s1[(size_t)a * N3 + e];
    if (b >= 0) v += s2[(size_t)b * N3 + e];
    d[e] = accumulate ? d[e] + v : v;
  }
}

// Transpose of cf_interp_kernel: the adjoint field on one fine block (mode 0),
// or the adjoint of the correction source on it (mode 1: first the transpose
// of the 7-point stencil onto the (N+2)^3 region, sign included), is spread
// back through the tensor-product quadratic weights onto the coarse region of
// the parent's 3x3x3 neighbourhood and added to the coarse field with atomics
// (neighbouring fine blocks share coarse cells).
template <typename R, int N, int MODE>
__global__ void __launch_bounds__(N >= 16 ? 256 : 128)
    cf_interp_adjoint_kernel(R* __restrict__ gcoarse, const int* __restrict__ nbr27, const R* __restrict__ gfine,
                             const int* __restrict__ fine_ids, const int* __restrict__ cposv,
                             const double* __restrict__ inv_hf2, int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int mode = MODE;
  constexpr int N3 = N * N * N;
  constexpr int halo = mode == 1 ? 1 : 0;
  constexpr int F = N + 2 * halo;
  constexpr int M = N / 2 + 2 + 2 * halo;
  R* C = reinterpret_cast<R*>(smem_raw);  // [M][M][M]
  R* T1 = C + M * M * M;                  // [M][M][F]
  R* T2 = T1 + M * M * F;                 // [M][F][F]
  R* U = T2 + M * F * F;                  // [F][F][F]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c = cposv[blockIdx.x];
  const int cp[3] = {c >> 2, (c >> 1) & 1, c & 1};
  int cbase[3];
  for (int a = 0; a < 3; ++a) cbase[a] = ((cp[a] * N - halo) >> 1) - 1;
  const R* g = gfine + (size_t)fine_ids[blockIdx.x] * N3;
  if (mode == 0) {
    for (int o = tid; o < N3; o += nt) U[o] = g[o];
  } else {
    const R ih2 = (R)inv_hf2[blockIdx.x];
    for (int o = tid; o < F * F * F; o += nt) {
      const int x[3] = {o / (F * F) - 1, (o / F) % F - 1, o % F - 1};  // fine index relative to the block
      auto in = [&](int i, int j, int k) { return i >= 0 && i < N && j >= 0 && j < N && k >= 0 && k < N; };
      auto gv = [&](int i, int j, int k) { return in(i, j, k) ? g[(i * N + j) * N + k] : R(0); };
      R v = gv(x[0] + 1, x[1], x[2]) + gv(x[0] - 1, x[1], x[2]) + gv(x[0], x[1] + 1, x[2]) + gv(x[0], x[1] - 1, x[2]) +
            gv(x[0], x[1], x[2] + 1) + gv(x[0], x[1], x[2] - 1) - R(6) * gv(x[0], x[1], x[2]);
      U[o] = -v * ih2;  // the correction subtracts the stencil
    }
  }
  __syncthreads();
  // transpose of the axis-0 pass: T2[ci][j][k] = sum_g w U[g][j][k]
  for (int o = tid; o < M * F * F; o += nt) {
    const int jk = o % (F * F), ci = o / (F * F);
    R s = 0;
    for (int gg = 0; gg < F; ++gg) {
      const int G = cp[0] * N + gg - halo, e = ci - ((G >> 1) - cbase[0]) + 1;
      if (e >= 0 && e < 3) s += cf_w<R>(G & 1, e) * U[gg * F * F + jk];
    }
    T2[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < M * M * F; o += nt) {  // axis 1
    const int k = o % F, cj = (o / F) % M, i = o / (M * F);
    R s = 0;
    for (int gg = 0; gg < F; ++gg) {
      const int G = cp[1] * N + gg - halo, e = cj - ((G >> 1) - cbase[1]) + 1;
      if (e >= 0 && e < 3) s += cf_w<R>(G & 1, e) * T2[(i * F + gg) * F + k];
    }
    T1[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < M * M * M; o += nt) {  // axis 2
    const int ck = o % M, ij = o / M;
    R s = 0;
    for (int gg = 0; gg < F; ++gg) {
      const int G = cp[2] * N + gg - halo, e = ck - ((G >> 1) - cbase[2]) + 1;
      if (e >= 0 && e < 3) s += cf_w<R>(G & 1, e) * T1[ij * F + gg];
    }
    C[o] = s;
  }
  __syncthreads();
  const int* nb = nbr27 + (size_t)blockIdx.x * 27;
  for (int o = tid; o < M * M * M; o += nt) {
    const R v = C[o];
    const int x[3] = {o / (M * M) + cbase[0], (o / M) % M + cbase[1], o % M + cbase[2]};
    int e[3], loc[3];
    for (int a = 0; a < 3; ++a) {
      e[a] = x[a] < 0 ? -1 : (x[a] >= N ? 1 : 0);
      loc[a] = x[a] - e[a] * N;
    }
    const int b = nb[(e[0] + 1) * 9 + (e[1] + 1) * 3 + (e[2] + 1)];
    if (b >= 0) {
      atomicAdd(&gcoarse[(size_t)b * N3 + (loc[0] * N + loc[1]) * N + loc[2]], v);
    } else if (v != R(0) && err_flag) {
      atomicExch(err_flag, 1);
    }
  }
}

// Transpose of the coarsening: every cell of the 8 children receives 1/8 of
// its coarse cell's adjoint, and the coarse (non-leaf) block is zeroed (its
// forward value was overwritten, so the user's value has zero gradient).
template <typename R>
__global__ void coarsen_adjoint_kernel(int N, R* __restrict__ g, const int* __restrict__ fine_ids,
                                       const int* __restrict__ coarse_ids) {
  const int N3 = N * N * N, H = N / 2;
  R* gc = g + (size_t)coarse_ids[blockIdx.x] * N3;
  for (int o = threadIdx.x; o < 8 * N3; o += blockDim.x) {
    const int a = o / N3, r = o % N3;
    const int i = r / (N * N), j = (r / N) % N, k = r % N;
    const int ci = (a >> 2) * H + i / 2, cj = ((a >> 1) & 1) * H + j / 2, ck = (a & 1) * H + k / 2;
    g[(size_t)fine_ids[blockIdx.x * 8 + a] * N3 + r] += R(0.125) * gc[(ci * N + cj) * N + ck];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < N3; o += blockDim.x) gc[o] = R(0);
}

template <typename R>
__global__ void laplacian_kernel(int N, const R* __restrict__ u, const int* __restrict__ nbr6, double inv_h2,
                                 R* __restrict__ out) {
  const int N3 = N * N * N;
  const int b = blockIdx.x;
  const int* nb = nbr6 + b * 6;  // (+0, -0, +1, -1, +2, -2)
  const R* ub = u + (size_t)b * N3;
  const R ih2 = (R)inv_h2;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int x[3] = {o / (N * N), (o / N) % N, o % N};
    R s = -R(6) * ub[o];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      for (int sg = 0; sg < 2; ++sg) {
        int y[3] = {x[0], x[1], x[2]};
        y[a] += sg == 0 ? 1 : -1;
        int blk = b;
        if (y[a] < 0 || y[a] >= N) {
          blk = nb[2 * a + sg];
          y[a] = (y[a] + N) % N;
        }
        if (blk < 0) { ok = false; continue; }
        s += u[(size_t)blk * N3 + (y[0] * N + y[1]) * N + y[2]];
      }
    }
    out[(size_t)b * N3 + o] = ok ? s * ih2 : R(0);
  }
}

// ---------------------------------------------------------------------------
static int threads_for(int N) { return N >= 16 ? 256 : 128; }

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Levels with at least kAnterpSeqParents parents (enough CTAs to fill the GPU
// without splitting parents) take one CTA per parent, the others a cluster of
// 8 CTAs per parent.
constexpr int kAnterpSeqParents = 2048;
template <typename R, int N, int NI>
static cudaError_t anterp_n(const double* J1, const int* parents, const int* children, int n, R* nodes, cudaStream_t s) {
  if (n >= kAnterpSeqParents)
    anterp_seq_kernel<R, N, NI><<<n, N * N, 0, s>>>(J1, parents, children, nodes);
  else
    anterp_kernel<R, N, NI><<<8 * n, N * N, 0, s>>>(J1, parents, children, nodes);  // clusters of 8 CTAs
  return cudaGetLastError();
}
template <typename R, int N, int NI>
static cudaError_t interp_n(const double* J1, const int* childs, const int* parents, const int* cpos, int n, R* unodes,
                            cudaStream_t s, bool compensated) {
  if constexpr (sizeof(R) == 4) {
    if (compensated) {
      interp_add_kernel<R, N, NI, ff><<<n, N * N, 0, s>>>(J1, childs, parents, cpos, unodes);
      return cudaGetLastError();
    }
  }
  interp_add_kernel<R, N, NI><<<n, N * N, 0, s>>>(J1, childs, parents, cpos, unodes);
  return cudaGetLastError();
}

// Dispatch over the supported (N, n_I): N in {8, 16}, 2 <= n_I <= min(N, 10).
#define FLGF_NI_CASES(N, F, ...)            \
  switch (nI) {                             \
    case 2: return F<R, N, 2>(__VA_ARGS__);  \
    case 3: return F<R, N, 3>(__VA_ARGS__);  \
    case 4: return F<R, N, 4>(__VA_ARGS__);  \
    case 5: return F<R, N, 5>(__VA_ARGS__);  \
    case 6: return F<R, N, 6>(__VA_ARGS__);  \
    case 7: return F<R, N, 7>(__VA_ARGS__);  \
    case 8: return F<R, N, 8>(__VA_ARGS__);  \
    default: break;                         \
  }

template <typename R>
cudaError_t launch_anterp(int N, int nI, const double* J1, const int* parents, const int* children, int n, R* nodes,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (N == 16) {
    FLGF_NI_CASES(16, anterp_n, J1, parents, children, n, nodes, s)
    if (nI == 9) return anterp_n<R, 16, 9>(J1, parents, children, n, nodes, s);
    if (nI == 10) return anterp_n<R, 16, 10>(J1, parents, children, n, nodes, s);
  } else if (N == 8) {
    FLGF_NI_CASES(8, anterp_n, J1, parents, children, n, nodes, s)
  }
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_interp_add(int N, int nI, const double* J1, const int* childs, const int* parents, const int* cpos,
                              int n, R* unodes, cudaStream_t s, bool compensated) {
  if (n <= 0) return cudaSuccess;
  if (N == 16) {
    FLGF_NI_CASES(16, interp_n, J1, childs, parents, cpos, n, unodes, s, compensated)
    if (nI == 9) return interp_n<R, 16, 9>(J1, childs, parents, cpos, n, unodes, s, compensated);
    if (nI == 10) return interp_n<R, 16, 10>(J1, childs, parents, cpos, n, unodes, s, compensated);
  } else if (N == 8) {
    FLGF_NI_CASES(8, interp_n, J1, childs, parents, cpos, n, unodes, s, compensated)
  }
  return cudaErrorInvalidValue;
}
#undef FLGF_NI_CASES

template <typename R>
cudaError_t launch_copy_blocks(int N, const R* src, const int* src_ids, R* dst, const int* dst_ids,
                               const uint8_t* zero, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  copy_blocks_kernel<R><<<n, threads_for(N), 0, s>>>(N, src, src_ids, dst, dst_ids, zero);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_coarsen(int N, const R* fine_f, const int* fine_ids, R* coarse_f, const int* coarse_ids, int n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  coarsen_kernel<R><<<n, threads_for(N), 0, s>>>(N, fine_f, fine_ids, coarse_f, coarse_ids);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cf_interp(int N, const R* ucoarse, const int* nbr27, const int* fine_ids, const int* cpos, int n,
                             R* fine, int mode, const double* inv_hf2, int* err_flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int halo = mode == 1 ? 1 : 0;
  const int F = N + 2 * halo, M = N / 2 + 2 + 2 * halo;
  const size_t sm = sizeof(R) * ((size_t)M * M * M + M * M * F + M * F * F + F * F * F);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<n, threads_for(N), sm, s>>>(ucoarse, nbr27, fine_ids, cpos, fine, inv_hf2, err_flag);
    return cudaSuccess;
  };
  cudaError_t e;
  if (N == 16) e = mode ? go(cf_interp_kernel<R, 16, 1>) : go(cf_interp_kernel<R, 16, 0>);
  else if (N == 8) e = mode ? go(cf_interp_kernel<R, 8, 1>) : go(cf_interp_kernel<R, 8, 0>);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_combine_blocks(int N, R* dst, const int* dst_ids, const R* s1, const int* s1_ids, const R* s2,
                                  const int* s2_ids, int accumulate, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  combine_blocks_kernel<R><<<n, threads_for(N), 0, s>>>(N, dst, dst_ids, s1, s1_ids, s2, s2_ids, accumulate);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cf_interp_adjoint(int N, R* gcoarse, const int* nbr27, const R* gfine, const int* fine_ids,
                                     const int* cpos, int n, int mode, const double* inv_hf2, int* err_flag,
                                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int halo = mode == 1 ? 1 : 0;
  const int F = N + 2 * halo, M = N / 2 + 2 + 2 * halo;
  const size_t sm = sizeof(R) * ((size_t)M * M * M + M * M * F + M * F * F + F * F * F);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<n, threads_for(N), sm, s>>>(gcoarse, nbr27, gfine, fine_ids, cpos, inv_hf2, err_flag);
    return cudaSuccess;
  };
  cudaError_t e;
  if (N == 16) e = mode ? go(cf_interp_adjoint_kernel<R, 16, 1>) : go(cf_interp_adjoint_kernel<R, 16, 0>);
  else if (N == 8) e = mode ? go(cf_interp_adjoint_kernel<R, 8, 1>) : go(cf_interp_adjoint_kernel<R, 8, 0>);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_coarsen_adjoint(int N, R* g, const int* fine_ids, const int* coarse_ids, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  coarsen_adjoint_kernel<R><<<n, threads_for(N), 0, s>>>(N, g, fine_ids, coarse_ids);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_laplacian(int N, const R* u, const int* nbr6, int n, double inv_h2, R* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  laplacian_kernel<R><<<n, threads_for(N), 0, s>>>(N, u, nbr6, inv_h2, out);
  return cudaGetLastError();
}

#define FLGF_INST(R)                                                                                            \
  template cudaError_t launch_anterp<R>(int, int, const double*, const int*, const int*, int, R*, cudaStream_t); \
  template cudaError_t launch_interp_add<R>(int, int, const double*, const int*, const int*, const int*, int, R*,       \
                                            cudaStream_t, bool);                                                \
  template cudaError_t launch_copy_blocks<R>(int, const R*, const int*, R*, const int*, const uint8_t*, int,    \
                                             cudaStream_t);                                                     \
  template cudaError_t launch_coarsen<R>(int, const R*, const int*, R*, const int*, int, cudaStream_t);         \
  template cudaError_t launch_cf_interp<R>(int, const R*, const int*, const int*, const int*, int, R*, int,     \
                                           const double*, int*, cudaStream_t);                                        \
  template cudaError_t launch_laplacian<R>(int, const R*, const int*, int, double, R*, cudaStream_t);            \
  template cudaError_t launch_combine_blocks<R>(int, R*, const int*, const R*, const int*, const R*, const int*, \
                                                int, int, cudaStream_t);                                        \
  template cudaError_t launch_cf_interp_adjoint<R>(int, R*, const int*, const R*, const int*, const int*, int,  \
                                                   int, const double*, int*, cudaStream_t);                     \
  template cudaError_t launch_coarsen_adjoint<R>(int, R*, const int*, const int*, int, cudaStream_t);
FLGF_INST(float)
FLGF_INST(double)

}  // namespace flgf
