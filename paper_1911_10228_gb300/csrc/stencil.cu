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
#include "common.cuh"
#include "internal.h"

namespace flgf {

template <typename R>
__global__ void anterp_kernel(int N, const double* __restrict__ J1, const int* __restrict__ parents,
                              const int* __restrict__ children, R* __restrict__ nodes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N3 = N * N * N;
  R* J = reinterpret_cast<R*>(smem_raw);  // [2N][N]
  R* A = J + 2 * N * N;
  R* B = A + N3;
  R* Pacc = B + N3;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 2 * N * N; i += nt) J[i] = (R)J1[i];
  for (int i = tid; i < N3; i += nt) Pacc[i] = R(0);
  const int parent = parents[blockIdx.x];
  for (int c = 0; c < 8; ++c) {
    const int cid = children[blockIdx.x * 8 + c];
    if (cid < 0) continue;
    const int c0 = c >> 2, c1 = (c >> 1) & 1, c2 = c & 1;
    __syncthreads();
    const R* src = nodes + (size_t)cid * N3;
    for (int i = tid; i < N3; i += nt) A[i] = src[i];
    __syncthreads();
    // axis 2: B[i][j][q] = sum_r J[c2 N + r][q] A[i][j][r]
    for (int o = tid; o < N3; o += nt) {
      const int q = o % N, ij = o / N;
      R s = 0;
      for (int r = 0; r < N; ++r) s += J[(c2 * N + r) * N + q] * A[ij * N + r];
      B[o] = s;
    }
    __syncthreads();
    // axis 1: A[i][q][k] = sum_r J[c1 N + r][q] B[i][r][k]
    for (int o = tid; o < N3; o += nt) {
      const int k = o % N, q = (o / N) % N, i = o / (N * N);
      R s = 0;
      for (int r = 0; r < N; ++r) s += J[(c1 * N + r) * N + q] * B[(i * N + r) * N + k];
      A[o] = s;
    }
    __syncthreads();
    // axis 0: Pacc[q][j][k] += sum_r J[c0 N + r][q] A[r][j][k]
    for (int o = tid; o < N3; o += nt) {
      const int jk = o % (N * N), q = o / (N * N);
      R s = 0;
      for (int r = 0; r < N; ++r) s += J[(c0 * N + r) * N + q] * A[r * N * N + jk];
      Pacc[o] += s;
    }
  }
  __syncthreads();
  R* dst = nodes + (size_t)parent * N3;
  for (int i = tid; i < N3; i += nt) dst[i] = Pacc[i];
}

template <typename R>
__global__ void interp_add_kernel(int N, const double* __restrict__ J1, const int* __restrict__ childs,
                                  const int* __restrict__ parents, const int* __restrict__ cpos,
                                  R* __restrict__ unodes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N3 = N * N * N;
  R* J = reinterpret_cast<R*>(smem_raw);
  R* A = J + 2 * N * N;
  R* B = A + N3;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 2 * N * N; i += nt) J[i] = (R)J1[i];
  const int child = childs[blockIdx.x], parent = parents[blockIdx.x], c = cpos[blockIdx.x];
  const int c0 = c >> 2, c1 = (c >> 1) & 1, c2 = c & 1;
  const R* src = unodes + (size_t)parent * N3;
  for (int i = tid; i < N3; i += nt) A[i] = src[i];
  __syncthreads();
  for (int o = tid; o < N3; o += nt) {  // axis 2
    const int r = o % N, ij = o / N;
    R s = 0;
    for (int q = 0; q < N; ++q) s += J[(c2 * N + r) * N + q] * A[ij * N + q];
    B[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < N3; o += nt) {  // axis 1
    const int k = o % N, r = (o / N) % N, i = o / (N * N);
    R s = 0;
    for (int q = 0; q < N; ++q) s += J[(c1 * N + r) * N + q] * B[(i * N + q) * N + k];
    A[o] = s;
  }
  __syncthreads();
  R* dst = unodes + (size_t)child * N3;
  for (int o = tid; o < N3; o += nt) {  // axis 0
    const int jk = o % (N * N), r = o / (N * N);
    R s = 0;
    for (int q = 0; q < N; ++q) s += J[(c0 * N + r) * N + q] * A[q * N * N + jk];
    dst[o] += s;
  }
}

template <typename R>
__global__ void copy_blocks_kernel(int N, const R* __restrict__ src, const int* __restrict__ src_ids,
                                   R* __restrict__ dst, const int* __restrict__ dst_ids,
                                   const uint8_t* __restrict__ zero) {
  const int N3 = N * N * N;
  const int i = blockIdx.x;
  const bool z = zero != nullptr && zero[i];
  const R* s = src + (size_t)src_ids[i] * N3;
  R* d = dst + (size_t)dst_ids[i] * N3;
  for (int e = threadIdx.x; e < N3; e += blockDim.x) d[e] = z ? R(0) : s[e];
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
__device__ __forceinline__ double cf_w(int sub, int e) {
  const double w0[3] = {5.0 / 32.0, 15.0 / 16.0, -3.0 / 32.0};
  return sub == 0 ? w0[e] : w0[2 - e];
}

template <typename R>
__global__ void cf_interp_kernel(int N, const R* __restrict__ ucoarse, const int* __restrict__ nbr27,
                                 const int* __restrict__ fine_ids, const int* __restrict__ cposv,
                                 R* __restrict__ fine, int mode, const double* __restrict__ inv_hf2, int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N3 = N * N * N;
  const int halo = mode == 1 ? 1 : 0;
  const int F = N + 2 * halo;       // fine region extent
  const int M = N / 2 + 2 + 2 * halo;  // coarse region extent
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
    for (int e = 0; e < 3; ++e) s += (R)cf_w(sub, e) * C[ij * M + ci + e - 1];
    T1[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < M * F * F; o += nt) {  // axis 1
    const int k = o % F, g = (o / F) % F, i = o / (F * F);
    const int G = cp[1] * N + g - halo, ci = (G >> 1) - cbase[1], sub = G & 1;
    R s = 0;
    for (int e = 0; e < 3; ++e) s += (R)cf_w(sub, e) * T1[(i * M + ci + e - 1) * F + k];
    T2[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < F * F * F; o += nt) {  // axis 0
    const int jk = o % (F * F), g = o / (F * F);
    const int G = cp[0] * N + g - halo, ci = (G >> 1) - cbase[0], sub = G & 1;
    R s = 0;
    for (int e = 0; e < 3; ++e) s += (R)cf_w(sub, e) * T2[(ci + e - 1) * F * F + jk];
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

template <typename R>
cudaError_t launch_anterp(int N, const double* J1, const int* parents, const int* children, int n, R* nodes,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = sizeof(R) * (2 * N * N + 3 * N * N * N);
  cudaError_t e = set_smem(anterp_kernel<R>, sm);
  if (e != cudaSuccess) return e;
  anterp_kernel<R><<<n, threads_for(N), sm, s>>>(N, J1, parents, children, nodes);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_interp_add(int N, const double* J1, const int* childs, const int* parents, const int* cpos,
                              int n, R* unodes, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = sizeof(R) * (2 * N * N + 2 * N * N * N);
  cudaError_t e = set_smem(interp_add_kernel<R>, sm);
  if (e != cudaSuccess) return e;
  interp_add_kernel<R><<<n, threads_for(N), sm, s>>>(N, J1, childs, parents, cpos, unodes);
  return cudaGetLastError();
}

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
  cudaError_t e = set_smem(cf_interp_kernel<R>, sm);
  if (e != cudaSuccess) return e;
  cf_interp_kernel<R><<<n, threads_for(N), sm, s>>>(N, ucoarse, nbr27, fine_ids, cpos, fine, mode, inv_hf2, err_flag);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_laplacian(int N, const R* u, const int* nbr6, int n, double inv_h2, R* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  laplacian_kernel<R><<<n, threads_for(N), 0, s>>>(N, u, nbr6, inv_h2, out);
  return cudaGetLastError();
}

#define FLGF_INST(R)                                                                                            \
  template cudaError_t launch_anterp<R>(int, const double*, const int*, const int*, int, R*, cudaStream_t);      \
  template cudaError_t launch_interp_add<R>(int, const double*, const int*, const int*, const int*, int, R*,    \
                                            cudaStream_t);                                                      \
  template cudaError_t launch_copy_blocks<R>(int, const R*, const int*, R*, const int*, const uint8_t*, int,    \
                                             cudaStream_t);                                                     \
  template cudaError_t launch_coarsen<R>(int, const R*, const int*, R*, const int*, int, cudaStream_t);         \
  template cudaError_t launch_cf_interp<R>(int, const R*, const int*, const int*, const int*, int, R*, int,     \
                                           const double*, int*, cudaStream_t);                                        \
  template cudaError_t launch_laplacian<R>(int, const R*, const int*, int, double, R*, cudaStream_t);
FLGF_INST(float)
FLGF_INST(double)

}  // namespace flgf
