// flgf_convolve_static: the exact block convolution without any device
// allocation.
//
// Who needs it: callers that must not allocate device memory while they
// compute -- code that runs inside a memory pool owned by another framework,
// latency-critical loops that cannot afford cudaMalloc's implicit
// synchronisation, or processes whose device memory is fully reserved up
// front.  The block-set API allocates its spectra at flgf_blockset_create;
// this entry point instead keeps its scratch (the forward and accumulated
// spectra and the launch lists) in one file-scope __device__ array of fixed
// size that every GPU loading the library holds until the process exits.
//
// It computes u = h^2 (G * f) over at most kStaticMaxBlocks blocks whose
// octree has a single level (all blocks within a 4 x 4 x 4 box aligned to
// even coordinates), so every pair is an exact zero-padded FFT convolution:
// the same forward FFT, spectrum multiply-accumulate and inverse FFT kernels
// as flgf_solve, with their scratch in the static array.
#include <algorithm>
#include <array>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/flgf.h"
#include "common.cuh"
#include "internal.h"

namespace {

using namespace flgf;

constexpr int kStaticMaxBlocks = 32;
constexpr size_t kSpecBytes = (size_t)kStaticMaxBlocks * nfreq(16) * 16;  // complex double, N = 16
constexpr size_t kListBytes = 512 * 1024;
constexpr size_t kScratchBytes = 2 * kSpecBytes + kListBytes;             // ~18.3 MB

// Shared by every call on a device; see the header for the concurrency rule.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (set up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Launch lists of one call, passed to the list-writing kernel by value (the
// kernel's parameters are copied at launch, so nothing is read from host
// memory afterwards).  At most 8 parents with targets and 8 neighbour cells
// with sources: the blocks lie in one aligned 4x4x4 box.
struct StaticLists {
  HadGroup group;
  int nchunk, nblk;
  double h2;
  int src[8 * 8];
  int tgt[8 * 8];
  uint16_t par[27 * 8];
};

// Offsets of the lists in the scratch array (256-byte aligned).
constexpr size_t kOffGroup = 0;
constexpr size_t kOffIds = 256;
constexpr size_t kOffScale = kOffIds + 256;
constexpr size_t kOffSrc = kOffScale + 256;
constexpr size_t kOffTgt = kOffSrc + 256;
constexpr size_t kOffPar = kOffTgt + 256;
constexpr size_t kOffWork = kOffPar + 512;

__global__ void static_lists_kernel(const StaticLists L, unsigned char* __restrict__ dl) {
  const int t = threadIdx.x;
  if (t == 0) *reinterpret_cast<HadGroup*>(dl + kOffGroup) = L.group;
  if (t < L.nblk) {
    reinterpret_cast<int*>(dl + kOffIds)[t] = t;
    reinterpret_cast<double*>(dl + kOffScale)[t] = L.h2;
  }
  if (t < 8 * L.group.ncell) reinterpret_cast<int*>(dl + kOffSrc)[t] = L.src[t];
  if (t < 8 * L.group.nact) reinterpret_cast<int*>(dl + kOffTgt)[t] = L.tgt[t];
  if (t < 27 * L.group.nact) reinterpret_cast<uint16_t*>(dl + kOffPar)[t] = L.par[t];
  // work items: (group 0, first chunk, chunks), cpc chunks each
  HadWork* w = reinterpret_cast<HadWork*>(dl + kOffWork);
  const int cpc = L.group.cpc;
  for (int i = t; i * cpc < L.nchunk; i += blockDim.x)
    w[i] = HadWork{0, i * cpc, min(cpc, L.nchunk - i * cpc)};
}

}  // namespace

extern "C" int flgf_convolve_static(flgf_ctx* ctx, int nblk, const int32_t* coords, const void* f, void* u,
                                    double h) {
  CtxView cv;
  if (!flgf::ctx_view(ctx, &cv)) return FLGF_EINVAL;
  auto bad = [&](int code, const char* m) {
    flgf::ctx_set_error(ctx, m);
    return code;
  };
  if (nblk < 1 || nblk > kStaticMaxBlocks || !coords || !f || !u || !(h > 0.0))
    return bad(FLGF_EINVAL, "convolve_static: need 1..32 blocks, coordinates, device f and u, h > 0");
  if (reinterpret_cast<uintptr_t>(f) % 16 || reinterpret_cast<uintptr_t>(u) % 16)
    return bad(FLGF_EINVAL, "convolve_static: f and u must be 16-byte aligned");
  const int N = cv.N;
  // one octree level: the parents of all blocks lie within one block of each other
  std::array<int, 3> plo = {INT32_MAX, INT32_MAX, INT32_MAX}, phi = {INT32_MIN, INT32_MIN, INT32_MIN};
  std::vector<std::array<int, 3>> c(nblk);
  for (int b = 0; b < nblk; ++b)
    for (int a = 0; a < 3; ++a) {
      c[b][a] = coords[3 * b + a];
      if (c[b][a] < -(1 << 19) || c[b][a] >= (1 << 19)) return bad(FLGF_EINVAL, "convolve_static: coordinate range");
      plo[a] = std::min(plo[a], c[b][a] >> 1);
      phi[a] = std::max(phi[a], c[b][a] >> 1);
    }
  for (int a = 0; a < 3; ++a)
    if (phi[a] - plo[a] > 1)
      return bad(FLGF_EINVAL, "convolve_static: blocks must lie in one 4x4x4 box aligned to even coordinates");
  {
    std::vector<std::array<int, 3>> s = c;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return bad(FLGF_EMESH, "convolve_static: duplicate block");
  }
  auto find = [&](int x, int y, int z) -> int {
    for (int b = 0; b < nblk; ++b)
      if (c[b][0] == x && c[b][1] == y && c[b][2] == z) return b;
    return -1;
  };
  // launch lists: one parent group over the parent box (one octree level,
  // near field included: every pair is a neighbour-parent pair)
  std::vector<ParentRec> recs;
  for (int p0 = plo[0]; p0 <= phi[0]; ++p0)
    for (int p1 = plo[1]; p1 <= phi[1]; ++p1)
      for (int p2 = plo[2]; p2 <= phi[2]; ++p2) {
        ParentRec r;
        bool has = false;
        for (int a = 0; a < 8; ++a) {
          r.tgt[a] = find(2 * p0 + (a >> 2), 2 * p1 + ((a >> 1) & 1), 2 * p2 + (a & 1));
          has |= r.tgt[a] >= 0;
        }
        if (!has) continue;
        for (int e = 0; e < 27; ++e)
          for (int b = 0; b < 8; ++b)
            r.cell[e][b] = find(2 * (p0 + e / 9 - 1) + (b >> 2), 2 * (p1 + (e / 3) % 3 - 1) + ((b >> 1) & 1),
                                2 * (p2 + e % 3 - 1) + (b & 1));
        recs.push_back(r);
      }
  const int nchunk = cv.fp64 ? nchunks<double>(N) : nchunks<float>(N);
  HadLists hl;
  pack_parent_groups(0, recs, nchunk, had_kernel_units(cv.fp64), hl);
  // one group of at most 8 parents and 8 cells (the parents lie in a 2x2x2 box)
  if (hl.groups.size() != 1 || hl.groups[0].nact > 8 || hl.groups[0].ncell > 8 ||
      kOffWork + sizeof(HadWork) * hl.work.size() > kListBytes)
    return bad(FLGF_EINVAL, "convolve_static: launch lists exceed the scratch");
  StaticLists L;
  std::memset(&L, 0, sizeof(L));
  L.group = hl.groups[0];
  L.nchunk = nchunk;
  L.nblk = nblk;
  L.h2 = h * h;
  std::copy(hl.src_ids.begin(), hl.src_ids.end(), L.src);
  std::copy(hl.tgt_ids.begin(), hl.tgt_ids.end(), L.tgt);
  std::copy(hl.par_tab.begin(), hl.par_tab.end(), L.par);

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return bad(FLGF_ECUDA, cudaGetErrorString(e));
  unsigned char* sp = static_cast<unsigned char*>(base);
  void* spec = sp;
  void* acc = sp + kSpecBytes;
  unsigned char* dl = sp + 2 * kSpecBytes;
  cudaStream_t s = cv.stream;
  // the lists travel as kernel parameters, written into the scratch on the stream
  static_lists_kernel<<<1, 256, 0, s>>>(L, dl);
  e = cudaGetLastError();
  const int* d_ids = reinterpret_cast<const int*>(dl + kOffIds);
  if (e == cudaSuccess) {
    if (cv.fp64) e = launch_fft_forward<double>(N, static_cast<const double*>(f), d_ids, d_ids, nblk, spec, nblk, s);
    else e = launch_fft_forward<float>(N, static_cast<const float*>(f), d_ids, d_ids, nblk, spec, nblk, s);
  }
  if (e == cudaSuccess) {
    const HadGroup* d_groups = reinterpret_cast<const HadGroup*>(dl + kOffGroup);
    const HadWork* d_work = reinterpret_cast<const HadWork*>(dl + kOffWork);
    const int* d_src = reinterpret_cast<const int*>(dl + kOffSrc);
    const int* d_tgt = reinterpret_cast<const int*>(dl + kOffTgt);
    const uint16_t* d_par = reinterpret_cast<const uint16_t*>(dl + kOffPar);
    const int nw = (int)hl.work.size();
    if (cv.fp64)
      e = launch_hadamard<double>(N, d_groups, d_work, nw, hl.max_units, d_src, d_tgt, d_par, spec, acc, nblk,
                                  cv.kspec, cv.kstride, s);
    else
      e = launch_hadamard<float>(N, d_groups, d_work, nw, hl.max_units, d_src, d_tgt, d_par, spec, acc, nblk,
                                 cv.kspec, cv.kstride, s);
  }
  if (e == cudaSuccess) {
    const double* d_scale = reinterpret_cast<const double*>(dl + kOffScale);
    if (cv.fp64) e = launch_fft_inverse<double>(N, acc, nblk, d_ids, d_ids, d_scale, nblk, static_cast<double*>(u), s, false);
    else e = launch_fft_inverse<float>(N, acc, nblk, d_ids, d_ids, d_scale, nblk, static_cast<float*>(u), s, false);
  }
  if (e != cudaSuccess) return bad(FLGF_ECUDA, cudaGetErrorString(e));
  return FLGF_OK;
}
