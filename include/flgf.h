/*
 * flgf.h -- C ABI of the GB300 (sm_103a) multi-resolution fast lattice
 * Green's function solver (Dorschner, Yu, Mengaldo & Colonius,
 * arXiv:1911.10228).
 *
 * Problem (Sec. 2, the discrete Poisson equation and Eq. discretConv):
 *     L_Q u(n) = f(n),  supp f in Omega_h,   u(n) = sum_m G(n - m) f(m),
 * with L_Q the 7-point Laplacian (sum of the 6 face neighbours minus 6 u)
 * and G its lattice Green's function on the unbounded lattice.  On a level
 * with spacing h the library returns u = h^2 (G * f), i.e. it solves
 * L_Q^{(h)} u = (7-point stencil)/h^2 u = f.
 *
 * Mesh (Sec. 2.1 and Sec. 3): a problem is a set of refinement levels
 * l = 0..L-1 (0 = coarsest, spacing h_l = h0 / 2^l).  Each level is a set of
 * cubic blocks of N^3 cells; block (c0, c1, c2) of level l covers cells
 * c*N .. c*N + N - 1 of that level's lattice on every axis.  Block c of level
 * l is refined ("non-leaf") when all 8 blocks 2c + {0,1}^3 exist on level
 * l+1; partial refinement is rejected.  Every non-leaf block must have its 26
 * same-level neighbours (the one-block buffer of Sec. 3, "Regularization and
 * Interpolation operators").  The answer is u on the leaf blocks of every
 * level; on non-leaf blocks the returned values are the field of the leaf
 * sources only (an intermediate of the scheme).
 *
 * Method: per level, the FLGF of Sec. 2.1 (octree of blocks, near field at
 * the finest octree level, influence lists, Lagrange interpolation with n_I
 * nodes, block-wise zero-padded (2N)^3 FFT convolution); across levels the
 * scheme of Sec. 3 (coarsening, two-FMM leaf/non-leaf subtraction,
 * accumulation with quadratic coarse-fine interpolation, source correction).
 *
 * Data layout: block values are arrays [nblk][N][N][N], C order (the last
 * index along axis 2 is fastest), in the order the blocks were given.
 * Values are double for FLGF_FP64 contexts and float for FLGF_FP32.
 *
 * Ownership: the library allocates and owns all device memory of a context
 * and a block set (allocation happens only in the *_create calls).  Pointers
 * passed in are borrowed for the duration of the call.  All GPU work is
 * enqueued on the context's stream; calls that read results into host memory
 * synchronise that stream.  A handle must not be used from two threads at
 * once; distinct handles are independent.
 *
 * Errors: every int-returning call returns FLGF_OK (0) or a negative FLGF_E*
 * code and never throws; flgf_last_error() describes the last failure of the
 * context.  A CUDA failure reports FLGF_ECUDA and may leave the context's
 * stream in an error state.
 */
#ifndef FLGF_H
#define FLGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FLGF_OK = 0,
  FLGF_EINVAL = -1,   /* bad argument (sizes, indices, precision, option) */
  FLGF_ENOMEM = -2,   /* device or host allocation failed */
  FLGF_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  FLGF_EMESH = -4,    /* block set violates the mesh rules (duplicates, partial refinement, buffer) */
  FLGF_ESTATE = -5,   /* call out of order (e.g. potential before solve) */
  FLGF_EDEVICE = -6   /* a kernel reported an error status (e.g. a missing halo block) */
};

enum { FLGF_FP64 = 0, FLGF_FP32 = 1 };  /* arithmetic and storage precision of a context */
enum { FLGF_HOST = 0, FLGF_DEVICE = 1 }; /* where a caller buffer lives */

typedef struct flgf_opts {
  int N;               /* block side, 8 or 16 (Sec. 2.1: blocks of N_b = n_b^3 cells) */
  int n_interp;        /* Lagrange interpolation nodes n_I, 2..min(N, 10) (Sec. 2.1) */
  int precision;       /* FLGF_FP64 or FLGF_FP32; LGF generation is always FP64 */
  int max_oct_levels;  /* octree levels whose kernel spectra are cached (1..8, default 6) */
  int table_radius;    /* LGF quadrature table radius, default 100 (Sec. 2) */
  int asym_radius;     /* A^3 up to this radius, A^2 beyond, default 600 (Sec. 2) */
  void* stream;        /* cudaStream_t for all work; NULL = the legacy default stream */
} flgf_opts;

typedef struct flgf_ctx flgf_ctx;
typedef struct flgf_blockset flgf_blockset;

/* Fill opts with the defaults above (N = 16, n_I = 6, FP64). */
void flgf_default_opts(flgf_opts* o);

/* Create a context: generates the FP64 LGF table by quadrature of Eq. GL_B
 * (|n| <= table_radius), the far-field switch (A^3, A^2; Sec. 2) and the
 * kernel spectra of every relative block offset in [-3, 3]^3 for octree
 * levels 0..max_oct_levels-1 (R2C FFT of the (2N)^3 kernel array
 * G(2^k (N d + Delta))).  Synchronises the stream.  *out is NULL on failure. */
int flgf_create(flgf_ctx** out, const flgf_opts* o);
void flgf_destroy(flgf_ctx* ctx);
/* Plan options of a context: they shape the launch lists of block sets
 * created afterwards (existing block sets keep theirs).  The paper has no
 * counterpart; they exist for tuning the spectrum multiply-accumulate:
 *   FLGF_CTX_LIST_PCT  0..100 (default 30): an interaction tile whose useful
 *                      (target, source) pairs are below this percentage of the
 *                      work of the dense parent-group kernel (8 x 8 children of
 *                      every neighbour parent pair, absent blocks included)
 *                      runs on the pair-list kernel instead; 0 = never.
 *   FLGF_CTX_TILE      tile in parents, t0 | t1 << 8 | t2 << 16 with
 *                      1 <= t_a <= 8, t0 t1 t2 <= 128 and
 *                      (t0 + 2)(t1 + 2)(t2 + 2) <= 397; default 4 x 4 x 8.
 *                      Tiles are the unit of the pair-list decision, and
 *                      their order is the order in which parents are packed
 *                      into the dense kernel's groups.
 *   FLGF_CTX_MAC       FP32 contexts: the kernels of the spectrum MAC.
 *                      1 (default): dense tiles with one target parent per
 *                      warp and two frequencies per thread (absent
 *                      cells and children are skipped warp-uniformly), sparse
 *                      tiles (FLGF_CTX_LIST_PCT) as pair lists with one target
 *                      per warp and one frequency per thread; 2: the same
 *                      dense kernel, sparse tiles in the shared-memory
 *                      pair-list kernel (one target per thread); 0: the
 *                      parent-group kernel (one parent per thread) and the
 *                      shared-memory pair-list kernel.  FP64 contexts always
 *                      use form 0; FLGF_CTX_ORDER applies to form 0 only.
 *   FLGF_CTX_ORDER     0 (default): the parents of each dense-kernel group keep
 *                      the tile order; 1: they are ordered by their set of
 *                      neighbours with sources (most first, equal sets
 *                      together), so the threads of a warp skip the same
 *                      absent neighbours (it loses the consecutive cell reads
 *                      of the tile order; measured slower on the uniform and
 *                      batched workloads, kept for the autotuner).
 *   FLGF_CTX_FAIL_ALLOC failure injection for tests of the error paths: with
 *                      value n >= 1 the n-th device allocation of the block
 *                      sets of this context (counted from this call; creation
 *                      and the adjoint's first use allocate) reports
 *                      FLGF_ENOMEM without allocating; 0 disarms.  One shot.
 * FLGF_EINVAL for an unknown key or a value out of range. */
enum { FLGF_CTX_LIST_PCT = 1, FLGF_CTX_TILE = 2, FLGF_CTX_FAIL_ALLOC = 3, FLGF_CTX_ORDER = 4, FLGF_CTX_MAC = 5 };
int flgf_ctx_set_option(flgf_ctx* ctx, int key, int value);

/* Message of the last failure on this context (never NULL; "" if none). */
const char* flgf_last_error(const flgf_ctx* ctx);

/* G(n) at n_pts integer points pts[3*i..3*i+2] as the library evaluates it
 * (table / A^3 / A^2), written to host memory out[n_pts].  Synchronises. */
int flgf_lgf_eval(flgf_ctx* ctx, int n_pts, const int32_t* pts, double* out);

/* Kernel spectrum of octree level k and block offset d = (d0, d1, d2) in
 * [-3, 3]^3, in natural order [k0 < 2N][k1 < 2N][k2 <= N] as interleaved
 * (re, im) doubles written to host memory out[2 * 4N^2(N+1)].  In FP32
 * contexts the stored single-precision values are widened.  Octree levels
 * k >= 1 never use the near offsets |d|_inf <= 1 (the near field belongs to
 * the finest level) and store them as zero.  Synchronises. */
int flgf_kernel_spectrum(flgf_ctx* ctx, int k, int d0, int d1, int d2, double* out);

/* Create a block set holding n_problems independent problems (1 for a plain
 * solve; several for the batched form, which runs every stage of all problems
 * in the same kernel launches).
 *   n_levels[p]              refinement levels of problem p (>= 1)
 *   nblk[q]                  blocks per level, concatenated over problems and levels
 *   coords[3*i..]            block coordinates, concatenated in the same order
 *   h0[p]                    spacing of level 0 of problem p (> 0)
 * Validates the mesh (FLGF_EMESH with a message on violation), builds each
 * level's octree, near/influence lists and launch tiles, and allocates all
 * device buffers. */
int flgf_blockset_create(flgf_ctx* ctx, int n_problems, const int* n_levels, const int* nblk,
                         const int32_t* coords, const double* h0, flgf_blockset** out);

/* As flgf_blockset_create, for a solve sharded over several GPUs by target
 * blocks (the multi-GPU form of Sec. 4's distribution of octants, with the
 * source replicated instead of exchanged): want[i] (one byte per block, in the
 * order of coords; NULL = every block) marks the blocks whose potential the
 * caller needs.  The block set then evaluates the far and near fields
 * (spectrum products, inverse FFTs, downward pass) only for those targets and
 * their octree ancestors; every (problem, level) source must still be loaded
 * in full.  The leaf-source fields that couple refinement levels (Sec. 3) are
 * computed for all blocks, so the potential on a wanted block equals that of
 * an unmasked solve; on other blocks it is unspecified.  Ranks that each
 * create a block set wanting a disjoint part (e.g. contiguous Morton-order
 * chunks) and gather their wanted blocks obtain the whole solution without
 * exchanging data during the solve.  want is borrowed for the call.  The
 * adjoint calls return FLGF_ESTATE on a block set that wants a subset. */
int flgf_blockset_create_masked(flgf_ctx* ctx, int n_problems, const int* n_levels, const int* nblk,
                                const int32_t* coords, const double* h0, const uint8_t* want,
                                flgf_blockset** out);
/* A vector Poisson problem (Sec. 3.1: the Cartesian components of the
 * streamfunction of a vorticity field, each a scalar problem on the same
 * mesh): n_components copies of one mesh (n_levels, nblk[n_levels], coords as
 * for one problem of flgf_blockset_create) as the problems 0 .. n_components-1
 * of one block set, problem c holding component c.  In an FP32 block set
 * (FLGF_CTX_MAC >= 1) the dense spectrum products of all components run in
 * the same CTAs, which stage the kernel spectra and the group tables once for
 * every component; the sums are the same, in the same order, as in
 * independent solves, so each component's potential equals its own scalar
 * solve bit for bit.  FP64 block sets solve the components as independent
 * problems of the block set.  1 <= n_components <= 64; arrays are borrowed
 * for the call. */
int flgf_blockset_create_vector(flgf_ctx* ctx, int n_components, int n_levels, const int* nblk,
                                const int32_t* coords, double h0, flgf_blockset** out);
void flgf_blockset_destroy(flgf_blockset* bs);

/* Total leaf cells (degrees of freedom of the composite mesh) over all problems. */
int64_t flgf_blockset_dof(const flgf_blockset* bs);

/* Copy the source of (problem, level) from f ([nblk][N][N][N], context
 * precision).  Values on non-leaf blocks are ignored (they are replaced by the
 * coarsened finer source, Sec. 3 step 1).
 * where = FLGF_HOST: the copy runs on the block set's own copy stream once the
 * last flgf_solve has taken its copy of the sources, so it overlaps the rest
 * of that solve; the call returns when the copy is done (f may be reused) and
 * the next flgf_solve waits for it.  A time-stepping caller can thus load
 * step i+1 before reading step i's potential.
 * where = FLGF_DEVICE: the copy is enqueued on the context stream (f must stay
 * valid until the next solve has run). */
int flgf_load_source(flgf_blockset* bs, int problem, int level, const void* f, int where);

/* Solve every problem of the block set (Sec. 3 algorithm; with one level it is
 * the FLGF of Sec. 2.1).  Enqueued on the context stream, no synchronisation. */
int flgf_solve(flgf_blockset* bs);

/* Copy u of (problem, level) into u ([nblk][N][N][N]).  Synchronises the
 * context stream (both forms) and returns FLGF_EDEVICE if a kernel of the last
 * solve raised the device error flag (a coarse-fine interpolation that met a
 * missing halo block); the flag is cleared at the start of every solve. */
int flgf_get_potential(flgf_blockset* bs, int problem, int level, void* u, int where);

/* One step of mesh generation on the device (Sec. 3.1, Eq. ref_crit: a block
 * of level l is refined where its source exceeds alpha^(L_R - l) times the
 * largest |source| on the level; Sec. 3: every refined block needs its 26
 * same-level neighbours).  Inputs on the device: f, the level's source
 * ([nblk][N][N][N], context precision), and coords ([nblk][3] int32 block
 * coordinates, |c| < 2^19); rel = alpha^(L_R - l) >= 0.  Outputs on the device:
 * flags[nblk] = 1 where max over the block of |f| > rel * (max over the level
 * of |f|), compared in FP64 (all 0 when the level's source is zero);
 * children[8 nblk][3] = the children (2c + {0,1}^3) of the flagged blocks, the
 * next level; buffer[26 nblk][3] = the 26-neighbours of flagged blocks that
 * are not blocks of the level, each once.  Both lists are in Morton order: by
 * the key interleaving the bits of (x, y, z) + 2^20 (bit i of x at key bit
 * 3i + 2, of y at 3i + 1, of z at 3i).  counts (host): {children, buffer}.
 * The call allocates its scratch (about 560 bytes per block) for its duration
 * and synchronises the context stream.  FLGF_EINVAL for a bad argument, a
 * coordinate out of range or nblk > 645277; FLGF_ENOMEM when the scratch
 * cannot be allocated.  The octree and interaction lists are still built on
 * the host by flgf_blockset_create. */
int flgf_refine_level(flgf_ctx* ctx, const void* f, int nblk, const int32_t* coords, double rel, uint8_t* flags,
                      int32_t* children, int32_t* buffer, int* counts);

/* out = L_Q^{(h_l)} u on the blocks of (problem, level), using same-level face
 * neighbours; cells with a missing neighbour get 0 (Sec. 3.1's consistency
 * check omega_h = L_Q Psi_h).  u and out: [nblk][N][N][N]. */
int flgf_laplacian(flgf_blockset* bs, int problem, int level, const void* u, void* out, int where);

/* Adjoint of the solve, for gradients (the paper has no adjoint; it follows
 * from the linear steps of Sec. 2.1 and Sec. 3).  The solve is linear,
 * u = A f with f the user sources of every (problem, level) (values on
 * non-leaf blocks ignored) and u the returned potentials; for adjoint seeds g
 * (one per (problem, level), [nblk][N][N][N], zero where the loss does not
 * look) flgf_solve_adjoint computes A^T g: the transposes of the correction,
 * accumulation, selection and coarsening steps in reverse order, and the FMMs
 * (symmetric: R = J^T and G(n) = G(-n)), the leaf-only one with its source
 * and target sets swapped.  The gradient of a loss with dL/du = g is then
 * dL/df = A^T g, zero on non-leaf blocks.  Seeds persist until reloaded; the
 * potentials of the last flgf_solve stay valid.
 * Enqueued on the context stream; the source correction option applies.  The
 * first flgf_load_adjoint or flgf_solve_adjoint of a block set builds its
 * adjoint lists and allocates the adjoint buffers (FLGF_ENOMEM on failure;
 * a later call retries).  flgf_get_gradient synchronises like
 * flgf_get_potential and reports the device error flag of the adjoint solve.
 * The transposed coarse-fine interpolation adds the contributions of
 * neighbouring fine blocks to shared coarse cells with atomic additions, so on
 * refined meshes the gradient is reproducible to round-off, not bit for bit. */
int flgf_load_adjoint(flgf_blockset* bs, int problem, int level, const void* g, int where);
int flgf_solve_adjoint(flgf_blockset* bs);
int flgf_get_gradient(flgf_blockset* bs, int problem, int level, void* out, int where);

/* Options of a block set. */
enum {
  FLGF_OPT_CORRECTION = 1,  /* 1 (default): source correction of Sec. 3 on; 0: off */
  FLGF_OPT_GRAPH = 2,       /* 1: capture the solve's launch sequence in a CUDA graph on first use */
  FLGF_OPT_TIMING = 3,      /* 1: record CUDA events between stages (see flgf_stage_times) */
  FLGF_OPT_COMPENSATED = 4, /* FP32 block sets: 1 runs the inverse FFTs of the octree levels above
                               the finest and the downward-pass interpolation in compensated
                               float-float arithmetic (about 48-bit significands on the FP32 pipes).
                               The interpolation extrapolates those levels' fields to the outer
                               faces of the child blocks, which amplifies FP32 rounding noise up to
                               ~38x at block corners (n_I = 6); compensation keeps refined meshes
                               within 1e-5 of the FP64 solve.  Default: 1 for block sets with a
                               problem of two or more refinement levels, else 0.  No effect in
                               FP64 contexts. */
  FLGF_OPT_FAULT_HALO = 5   /* failure injection for tests (value 1): one coarse neighbour entry of
                               the first coarse-fine interpolation list is marked absent, as if the
                               mesh lacked that halo block; the following solve reads zero there and
                               flgf_get_potential returns FLGF_EDEVICE.  Irreversible: the block
                               set's results are wrong from then on. */
};
int flgf_set_option(flgf_blockset* bs, int key, int value);

/* Stage times in ms accumulated over the solves run with FLGF_OPT_TIMING = 1
 * since the last reset, and the number of solves.  Stages:
 * 0 coarsen, 1 anterpolation, 2 forward FFT, 3 spectrum MAC, 4 inverse FFT,
 * 5 interpolation, 6 multi-resolution coupling (select, J^l, correction).
 * n_stages <= 7.  reset != 0 zeroes the accumulators afterwards. */
int flgf_stage_times(flgf_blockset* bs, double* ms, int n_stages, int* n_solves, int reset);

/* Work of one solve for roofline accounting: the number of (target, source)
 * block pairs of the spectrum MAC, of forward and inverse FFTs and of cached
 * kernel-spectrum offsets it touches. */
int flgf_work_counts(const flgf_blockset* bs, int64_t* pairs, int64_t* fwd_ffts, int64_t* inv_ffts,
                     int64_t* kernel_offsets);

/* Exact block convolution without device allocation: u = h^2 (G * f) over
 * nblk <= 32 blocks of N^3 cells whose parents (c >> 1) lie within one block
 * of each other on every axis (a 4x4x4 box aligned to even coordinates), so
 * every (target, source) pair is a zero-padded FFT convolution with no
 * interpolation.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory while they compute (code inside
 * another framework's memory pool, latency-critical loops that must avoid
 * cudaMalloc's implicit synchronisation, processes whose device memory is
 * reserved up front).
 *   coords  host array [nblk][3] of block coordinates
 *   f, u    DEVICE arrays [nblk][N][N][N] in the context precision (borrowed),
 *           16-byte aligned
 *   h       lattice spacing (> 0)
 * Scratch: the spectra and launch lists live in a fixed ~18 MB array in
 * device memory that the library declares statically; every GPU that loads
 * the library holds it until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress); make that
 * first call outside any stream capture.  The call allocates nothing (no
 * cudaMalloc or cudaFree), enqueues its work on the context stream and does
 * not synchronise: its launch lists travel as the parameters of a small
 * kernel that writes them into the array, so nothing is read from host memory
 * after the call returns.  The library cannot check the sizes of f and u:
 * they must hold nblk blocks.  All calls on a device share the array, so calls whose
 * GPU work may overlap (several contexts or streams on the same device) race;
 * serialise them.  Returns FLGF_EINVAL for more than 32 blocks or blocks
 * outside one aligned 4x4x4 box, FLGF_EMESH for duplicate blocks. */
int flgf_convolve_static(flgf_ctx* ctx, int nblk, const int32_t* coords, const void* f, void* u, double h);

/* Number of kernels the last flgf_solve enqueued (one per launch; a replayed
 * CUDA graph launches the same kernels as the solve it captured). */
int64_t flgf_launch_count(const flgf_blockset* bs);

#ifdef __cplusplus
}
#endif

#endif /* FLGF_H */
