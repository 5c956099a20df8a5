// a0: lattice Green's function table and per-offset kernel arrays (FP64).
//
// Sec. 2: G is tabulated by quadrature of Eq. GL_B for |n| <= 100 (Euclidean
// norm), the three-term far-field expansion A^3 is used for 100 < |n| <= 600
// and the two-term A^2 beyond.  The quadrature (exp-sinh rule, Miller/Hankel
// Bessel values) is in lgf_math.cuh.  The table stores only canonical points
// n1 >= n2 >= n3 >= 0; G has the 48-fold symmetry of the cubic lattice.
#include "common.cuh"
#include "internal.h"
#include "lgf_math.cuh"

namespace flgf {

int quad_nodes() { return kQuadNodes; }

// One thread per quadrature node: ive(k, 2 t_j) for k = 0..K into B[k][j];
// row K+1 receives the quadrature weight of node j.
__global__ void bessel_table_kernel(double* __restrict__ B, int K) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kQuadNodes) return;
  ive_orders(2.0 * de_node_t(j), K, B + j, kQuadNodes);
  B[(size_t)(K + 1) * kQuadNodes + j] = de_node_w(j);
}

cudaError_t launch_bessel_table(double* B, int K, cudaStream_t s) {
  bessel_table_kernel<<<(kQuadNodes + 127) / 128, 128, 0, s>>>(B, K);
  return cudaGetLastError();
}

__device__ __forceinline__ size_t tab_idx(int a, int b, int c, int R) {
  return ((size_t)a * (R + 1) + b) * (R + 1) + c;
}

// One thread per canonical point: G = - sum_j w_j ive(a,2t_j) ive(b,2t_j) ive(c,2t_j).
__global__ void lgf_table_kernel(const double* __restrict__ B, int K, double* __restrict__ table, int R) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int side = R + 1;
  if (idx >= side * side * side) return;
  const int a = idx / (side * side), b = (idx / side) % side, c = idx % side;
  if (!(a >= b && b >= c)) return;
  if ((double)a * a + (double)b * b + (double)c * c > (double)R * R) return;
  const double* Ba = B + (size_t)a * kQuadNodes;
  const double* Bb = B + (size_t)b * kQuadNodes;
  const double* Bc = B + (size_t)c * kQuadNodes;
  const double* W = B + (size_t)(K + 1) * kQuadNodes;
  double s = 0.0;
  for (int j = 0; j < kQuadNodes; ++j) s += W[j] * (Ba[j] * Bb[j] * Bc[j]);
  table[tab_idx(a, b, c, R)] = -s;
}

cudaError_t launch_lgf_table(const double* B, int K, double* table, int R, cudaStream_t s) {
  if (K < R) return cudaErrorInvalidValue;
  const int total = (R + 1) * (R + 1) * (R + 1);
  lgf_table_kernel<<<(total + 255) / 256, 256, 0, s>>>(B, K, table, R);
  return cudaGetLastError();
}

// G at an arbitrary lattice point with the table / A^3 / A^2 switch.
__device__ double lgf_at(const double* __restrict__ table, int R, double rt2, double ra2, long long n0,
                         long long n1, long long n2) {
  long long a = n0 < 0 ? -n0 : n0, b = n1 < 0 ? -n1 : n1, c = n2 < 0 ? -n2 : n2;
  // sort descending: a >= b >= c
  if (a < b) { long long t = a; a = b; b = t; }
  if (b < c) { long long t = b; b = c; c = t; }
  if (a < b) { long long t = a; a = b; b = t; }
  const double r2 = (double)a * a + (double)b * b + (double)c * c;
  if (r2 <= rt2) return table[tab_idx((int)a, (int)b, (int)c, R)];
  if (r2 <= ra2) return lgf_asym3((double)a, (double)b, (double)c);
  return lgf_asym2((double)a, (double)b, (double)c);
}

__global__ void lgf_eval_kernel(const double* __restrict__ table, int R, double rt2, double ra2,
                                const int32_t* __restrict__ pts, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = lgf_at(table, R, rt2, ra2, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
}

cudaError_t launch_lgf_eval(const double* table, int R, double rt, double ra, const int32_t* pts, int n,
                            double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  lgf_eval_kernel<<<(n + 255) / 256, 256, 0, s>>>(table, R, rt * rt, ra * ra, pts, n, out);
  return cudaGetLastError();
}

__global__ void kernel_arrays_kernel(const double* __restrict__ table, int R, double rt2, double ra2, int N,
                                     int k, double* __restrict__ out) {
  const int P = 2 * N;
  const size_t per = (size_t)P * P * P;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per * kNOff) return;
  const int d = (int)(idx / per);
  const int rem = (int)(idx % per);
  const int i0 = rem / (P * P), i1 = (rem / P) % P, i2 = rem % P;
  if (i0 == N || i1 == N || i2 == N) { out[idx] = 0.0; return; }
  const int d0 = d / 49 - 3, d1 = (d / 7) % 7 - 3, d2 = d % 7 - 3;
  const long long s = 1LL << k;
  const long long x0 = s * ((long long)N * d0 + (i0 < N ? i0 : i0 - P));
  const long long x1 = s * ((long long)N * d1 + (i1 < N ? i1 : i1 - P));
  const long long x2 = s * ((long long)N * d2 + (i2 < N ? i2 : i2 - P));
  out[idx] = lgf_at(table, R, rt2, ra2, x0, x1, x2);
}

cudaError_t launch_kernel_arrays(const double* table, int R, double rt, double ra, int N, int k, double* out,
                                 cudaStream_t s) {
  const size_t total = (size_t)kNOff * (2 * N) * (2 * N) * (2 * N);
  kernel_arrays_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(table, R, rt * rt, ra * ra, N, k, out);
  return cudaGetLastError();
}

}  // namespace flgf
