// Internal launcher interface between the host orchestration (flgf_api.cu)
// and the kernels (lgf.cu, fft.cu, hadamard.cu, hadamard_fl.cu, stencil.cu,
// meshgen.cu, flgf_static.cu).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

struct flgf_ctx;

namespace flgf {

// Read-only view of a context (defined in flgf_api.cu).
struct CtxView {
  int N;
  bool fp64;
  cudaStream_t stream;
  const void* kspec;  // [octree level][chunk][343][T]
  size_t kstride;     // complex elements per octree level
};
bool ctx_view(const flgf_ctx* c, CtxView* v);
void ctx_set_error(flgf_ctx* c, const char* msg);

// ---- a0: LGF table and kernel arrays (lgf.cu) ----------------------------
// Bessel table B[k][j] = ive(k, 2 t_j), k = 0..K, j over the exp-sinh nodes.
cudaError_t launch_bessel_table(double* B, int K, cudaStream_t s);
int quad_nodes();
// Canonical LGF table T[n1][n2][n3] (0 <= n3 <= n2 <= n1 <= R, n1^2+n2^2+n3^2 <= R^2).
cudaError_t launch_lgf_table(const double* B, int K, double* table, int R, cudaStream_t s);
// LGF at integer points pts[i] (x3) with the table / A^3 / A^2 switch.
cudaError_t launch_lgf_eval(const double* table, int R, double rt, double ra, const int32_t* pts,
                            int n, double* out, cudaStream_t s);
// (2N)^3 circular kernel arrays for octree level k, every offset d in [-3,3]^3:
// out[d][i0][i1][i2] = G(2^k (N d + Delta)), Delta = i (i < N) or i - 2N (i > N), 0 at i == N.
cudaError_t launch_kernel_arrays(const double* table, int R, double rt, double ra, int N, int k,
                                 double* out, cudaStream_t s);

// ---- a2/a4 FFTs (fft.cu) ---------------------------------------------------
cudaError_t fft_init_constants();
// Forward R2C of zero-padded N^3 blocks: in[gid_list[i]] -> spec column sid_list[i].
template <typename R>
cudaError_t launch_fft_forward(int N, const R* nodes, const int* gids, const int* sids, int count,
                               void* spec, int spec_blocks, cudaStream_t s);
// Inverse C2R, keep the first N^3 outputs, scale by scale[i]/(2N)^3, write (or add) to out[gids[i]].
// compensated: FP32 spectra transformed in float-float arithmetic (ffloat.cuh).
template <typename R>
cudaError_t launch_fft_inverse(int N, const void* acc, int spec_blocks, const int* sids, const int* gids,
                               const double* scales, int count, R* out, cudaStream_t s, bool compensated);
// Kernel spectra of one octree level from the (2N)^3 kernel arrays (FP64 FFT),
// stored as [chunk][343][T] in precision R; zero_near stores the 27 near
// offsets as zero (octree levels >= 1 never use them).
template <typename R>
cudaError_t launch_kernel_spectra(int N, const double* karr, void* kspec_level, double* tmp, int zero_near,
                                  cudaStream_t s);

// ---- a3 spectrum multiply-accumulate (hadamard.cu) ------------------------
// Dense MAC: groups of parents (see hadamard.cu).
struct HadGroup {
  int level;     // octree level k (selects the kernel spectra)
  int nact;      // parents (<= kHadMaxParents)
  int pslots;    // parent slots per (frequency group, chunk): power of two >= nact
  int cpc;       // frequency chunks per CTA (pslots * 2 * cpc <= kHadThreads threads)
  int ncell;     // neighbour cells that hold sources
  int par_off;   // into the parent table: [27][nact] cell of neighbour e, or kNbEnd
  int tgt_off;   // into the target list: [nact][8] spectrum column or -1 (child a = 4 a0 + 2 a1 + a2)
  int src_off;   // into the source list: [8][ncell] spectrum column of child b of cell c, or -1
};
// Work item of the dense MAC: (group, first chunk, chunks).
struct HadWork {
  int group, chunk0, nch;
};
constexpr int kHadThreads = 256;              // threads per CTA
constexpr int kHadMaxCpc = 4;                 // frequency chunks per CTA
constexpr int kHadMaxParents = 128;           // parents per group
constexpr size_t kHadSmemBytes = 110 * 1024;  // dynamic shared memory per CTA (two CTAs per SM)
constexpr uint16_t kNbEnd = 0xFFFF;           // no neighbour cell (cells < 2048)
// One parent with targets: its 8 children (spectrum column or -1) and, per
// neighbour e (e = 9 (e0+1) + 3 (e1+1) + (e2+1)), the 8 children of parent
// p + e that are sources (all -1 when there are none or the pair is excluded).
struct ParentRec {
  int tgt[8];
  int cell[27][8];
};
// Launch lists of the dense MAC, appended to by pack_parent_groups.
struct HadLists {
  std::vector<HadGroup> groups;
  std::vector<HadWork> work;
  std::vector<int> src_ids, tgt_ids;
  std::vector<uint16_t> par_tab;
  int max_units = 0;  // max over groups of their shared memory in 32-byte units
};
// Packs parent records, in order, into groups of one octree level and their
// work items (nchunk frequency chunks); kunits = 32-byte units of kernel
// spectra per chunk in shared memory (had_kernel_units).  order_by_list
// orders each group's parents by their set of neighbours with sources (most
// first, equal sets together) instead of keeping the record order.
void pack_parent_groups(int level, const std::vector<ParentRec>& recs, int nchunk, int kunits, HadLists& L,
                        bool order_by_list = false);
// Kernel-spectrum shared memory per chunk of the dense MAC, in 32-byte units:
// the complex values (FP32) or the three-product form (FP64, twice as large).
constexpr int had_kernel_units(bool fp64) { return fp64 ? 2 * kNOff : kNOff; }
template <typename R>
cudaError_t launch_hadamard(int N, const HadGroup* groups, const HadWork* work, int nwork, int max_units,
                            const int* src_ids, const int* tgt_ids, const uint16_t* par_tab, const void* spec, void* acc,
                            int spec_blocks, const void* kspec, size_t kspec_level_stride, cudaStream_t s);
// Sparse tiles: explicit (target, source) pair lists.  The targets of the
// sparse tiles of one octree level are pooled in tile order and cut into
// groups of up to kListTargets targets (sorted by list length within a group)
// whose source union fits shared memory; per target the pair entries are
// (local source slot << 9 | kernel offset index), stored entry-major
// [entry][kListTargets] so a warp reads consecutive words.
constexpr int kListTargets = 128;
constexpr int kListMaxSrc = 1400;  // sources per group: (343 + 1400) x 32 B of shared memory
struct ListGroup {
  int level;     // octree level (kernel spectra)
  int ntgt;      // targets in the group (<= kListTargets)
  int maxlen;    // longest pair list
  int tgt_off;   // into the target list: spectrum column per target
  int len_off;   // into the length list: pairs per target
  int ent_off;   // into the entry list: maxlen * kListTargets words
  int src_off;   // into the source list: spectrum column per local source slot
  int nsrc;
};
template <typename R>
cudaError_t launch_hadamard_list(int N, const ListGroup* groups, int ngroups, int max_src, const int* tgt,
                                 const int* len, const int* ent, const int* src, const void* spec, void* acc,
                                 int spec_blocks, const void* kspec, size_t kspec_level_stride, cudaStream_t s);

// FP32 frequency-lane MAC (hadamard_fl.cu): a CTA takes a group of at most
// kFlMaxParents consecutive target parents (with at most kFlMaxCells
// neighbour cells) and a block of kFlFreq consecutive frequencies; a warp
// owns one parent, a lane two consecutive frequencies.  Per parent a row of kFlRowStride
// uint16: [0] = number of cells n, [1 .. n] = e << 11 | cell for its
// neighbours e with products, in increasing e; cell indexes the group's cell
// table of the 8 children's spectrum columns (-1 where a child is no source).
// Beside it kFlDelta uint32 delta masks, entry j for row entry 1 + j: bit
// ((l0 + 1) * 3 + l1 + 1) * 3 + l2 + 1 set when a target-source child pair
// with a - b = l contributes, bit 31 when all 27 may run (fl_delta_mask).
constexpr int kFlWarps = 16;
constexpr int kFlMaxParents = 128;
constexpr int kFlMaxCells = 768;
constexpr int kFlFreq = 64;
constexpr int kFlRowStride = 28;
constexpr int kFlDelta = kFlRowStride - 1;
constexpr size_t kFlSmemBytes = 227 * 1024;  // one CTA per SM
struct FlGroup {
  int level;     // octree level (kernel spectra)
  int nact;      // target parents
  int ncell;     // neighbour cells with sources
  int row_off;   // first parent: rows [row_off + m][kFlRowStride], targets [row_off + m][8]
  int cell_off;  // first cell: [cell_off + c][8]
};
struct FlLists {
  std::vector<FlGroup> groups;
  std::vector<uint16_t> rows;  // [parents][kFlRowStride]
  std::vector<uint32_t> dlms;  // [parents][kFlDelta] delta masks of the row entries
  std::vector<int> tgt_ids;    // [parents][8] spectrum column or -1
  std::vector<int> cells;      // [cells][8] spectrum column or -1
  int max_cells = 0, max_parents = 0;
};
// Packs parent records, in order, into frequency-lane groups of one octree level.
void pack_fl_groups(int level, const std::vector<ParentRec>& recs, FlLists& L);
uint32_t fl_delta_mask(int level, int e, const int* tgt, const int* src);
size_t fl_smem_bytes(int max_cells, int max_parents);
// ncomp > 1: a vector block set's components, whose spectrum columns are
// component 0's + c * cstride, run through the same groups in one launch.
cudaError_t launch_hadamard_fl(int N, const FlGroup* groups, int ngroups, int max_cells, int max_parents,
                               const uint16_t* rows, const uint32_t* dlms, const int* tgt_ids, const int* cells,
                               const void* spec, void* acc, int spec_blocks, const void* kspec,
                               size_t kspec_level_stride, int ncomp, int cstride, bool split, cudaStream_t s);
// Full rows at or above this fraction of a phase's rows: the two-path product form.
constexpr double kFlSplitFullFraction = 0.9;
// FP32 frequency-lane pair lists (hadamard_fl.cu), for the targets of sparse
// tiles: a CTA takes a group of at most kFllTargets targets and a block of
// kFllFreq consecutive frequencies, a warp one target at a time, a lane one
// frequency.  Target i of the phase has its spectrum column tgt[i] and the
// entries ent[beg[i] .. beg[i] + len[i]) = source column << 9 | kernel offset
// index (the pair-list pool's own format).
constexpr int kFllWarps = 16;
constexpr int kFllFreq = 32;
constexpr int kFllTargets = 64;
struct FllGroup {
  int level;    // octree level (kernel spectra)
  int ntgt;     // targets (<= kFllTargets), longest list first
  int tgt_off;  // first target index
};
struct FllLists {
  std::vector<FllGroup> groups;
  std::vector<int> tgt, beg, len;
  std::vector<uint32_t> ent;
};
// Packs the pair-list pool of one octree level, in order, into groups.
void pack_fll_groups(int level, const std::vector<std::pair<int, std::vector<int>>>& pool, FllLists& L);
cudaError_t launch_hadamard_fll(int N, const FllGroup* groups, int ngroups, const int* tgt, const int* beg,
                                const int* len, const uint32_t* ent, const void* spec, void* acc, int spec_blocks,
                                const void* kspec, size_t kspec_level_stride, cudaStream_t s);


// ---- on-device refinement of a level (meshgen.cu) ----------------------------
// f: [nblk][N^3] in the context precision; coords, flags, children, buffer on
// the device, counts on the host (see flgf_refine_level).  cudaErrorInvalidValue
// for a coordinate outside (-2^19, 2^19) or more than 2^24 / 26 blocks.
cudaError_t launch_refine_level(int N, int prec_fp64, const void* f, int nblk, const int32_t* coords, double rel,
                                uint8_t* flags, int32_t* children, int32_t* buffer, int* counts, cudaStream_t s);

// ---- a1/a5 and multi-resolution stencils (stencil.cu) ----------------------
// J1: dense 1-D Lagrange matrix [2N][N] (row = child node of the two children, column = parent node).
template <typename R>
cudaError_t launch_anterp(int N, int nI, const double* J1, const int* parents, const int* children /*[n][8]*/,
                          int n, R* nodes, cudaStream_t s);
template <typename R>
// compensated: FP32 data interpolated in float-float arithmetic (ffloat.cuh).
cudaError_t launch_interp_add(int N, int nI, const double* J1, const int* childs, const int* parents, const int* cpos,
                              int n, R* unodes, cudaStream_t s, bool compensated);
// dst[dst_ids[i]] = src[src_ids[i]] * (mask? mask[i] : 1)
template <typename R>
cudaError_t launch_copy_blocks(int N, const R* src, const int* src_ids, R* dst, const int* dst_ids,
                               const uint8_t* zero, int n, cudaStream_t s);
// Coarsening: out[coarse[i]] = mean of 8 fine cells of children fine[i][8]
template <typename R>
cudaError_t launch_coarsen(int N, const R* fine_f, const int* fine_ids, R* coarse_f, const int* coarse_ids,
                           int n, cudaStream_t s);
// Coarse-fine quadratic interpolation from level l to level l+1 blocks.
// nbr27[i][27]: coarse block ids of the parent's 3x3x3 neighbourhood (-1 if absent);
// mode 0: ufine[fine[i]] += J u_coarse; mode 1: ffine[fine[i]] -= L^{(hf)} J u_coarse, inv_hf2[i] = 1/hf^2.
template <typename R>
cudaError_t launch_cf_interp(int N, const R* ucoarse, const int* nbr27, const int* fine_ids, const int* cpos,
                             int n, R* fine, int mode, const double* inv_hf2, int* err_flag, cudaStream_t s);
// Adjoint operators: dst[i] (+)= s1[i] + s2[i] (ids < 0 contribute nothing);
// transpose of launch_cf_interp (scatter-add onto the coarse field); transpose
// of the coarsening (spread 1/8 to the children, zero the coarse block).
template <typename R>
cudaError_t launch_combine_blocks(int N, R* dst, const int* dst_ids, const R* s1, const int* s1_ids, const R* s2,
                                  const int* s2_ids, int accumulate, int n, cudaStream_t s);
template <typename R>
cudaError_t launch_cf_interp_adjoint(int N, R* gcoarse, const int* nbr27, const R* gfine, const int* fine_ids,
                                     const int* cpos, int n, int mode, const double* inv_hf2, int* err_flag,
                                     cudaStream_t s);
template <typename R>
cudaError_t launch_coarsen_adjoint(int N, R* g, const int* fine_ids, const int* coarse_ids, int n, cudaStream_t s);
// 7-point Laplacian with same-level face neighbours nbr6[i][6] (-1 absent -> 0 output).
template <typename R>
cudaError_t launch_laplacian(int N, const R* u, const int* nbr6, int n, double inv_h2, R* out, cudaStream_t s);

}  // namespace flgf
