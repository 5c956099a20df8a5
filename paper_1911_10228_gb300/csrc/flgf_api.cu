// Host side of the FLGF library: context set-up (LGF table, kernel spectra),
// block-set compilation (mesh checks, octrees, interaction tiles, parent groups
// and pair lists, launch lists), the solve sequence of Sec. 2.1 / Sec. 3 and
// its adjoint.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/flgf.h"
#include "common.cuh"
#include "internal.h"

using namespace flgf;

struct flgf_ctx {
  int N = 16, nI = 6, prec = FLGF_FP64, max_oct = 6, R = 100, RA = 600;
  // plan options for block sets created afterwards (flgf_ctx_set_option)
  int list_pct = 30;             // pair-list MAC below this useful fraction of the dense kernel's work
  int tile[3] = {4, 4, 8};       // dense MAC tile in parents
  bool order_by_list = false;    // dense MAC groups: parents ordered by neighbour set (FLGF_CTX_ORDER)
  int mac = 1;                   // FP32 MAC form (FLGF_CTX_MAC): 1 frequency-lane (dense and lists), 2 frequency-lane
                                 // dense + shared-memory lists, 0 parent groups + shared-memory lists
  // failure injection (FLGF_CTX_FAIL_ALLOC): the fail_alloc_at-th block-set
  // device allocation from the arming on reports out-of-memory instead of allocating
  int fail_alloc_at = 0, alloc_count = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  double* d_table = nullptr;
  double* d_J1 = nullptr;
  void* d_kspec = nullptr;
  size_t kstride = 0;  // complex elements per octree level
  std::vector<double> J1;
};

namespace {

using I3 = std::array<int, 3>;

int fail(flgf_ctx* c, int code, const std::string& m) {
  if (c) c->err = m;
  return code;
}

// Device allocation of block-set buffers (at least 256 bytes), with the
// failure-injection hook of FLGF_CTX_FAIL_ALLOC.
cudaError_t dev_alloc(flgf_ctx* ctx, void** p, size_t bytes) {
  if (ctx->fail_alloc_at > 0 && ++ctx->alloc_count == ctx->fail_alloc_at) {
    ctx->fail_alloc_at = 0;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, std::max<size_t>(bytes, 256));
}

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

inline uint64_t key3(int a, int b, int c) {
  const uint64_t o = 1u << 20;
  return ((uint64_t)(a + o) << 42) | ((uint64_t)(b + o) << 21) | (uint64_t)(c + o);
}
inline uint64_t key3(const I3& v) { return key3(v[0], v[1], v[2]); }

// 1-D Lagrange interpolation between octree levels (Sec. 2.1).  A level-k
// block's nodes are the centres of its N cells: in units of the child
// spacing the 2N nodes of two sibling children lie at j + 1/2 and the N
// parent nodes at 2p + 1.  Each child node takes the n_I parent nodes nearest
// to it (window centred on it, moved inwards at the faces).
std::vector<double> lagrange_matrix(int N, int nI) {
  std::vector<double> J((size_t)2 * N * N, 0.0);
  for (int j = 0; j < 2 * N; ++j) {
    const double x = j + 0.5;
    int start;
    if (nI % 2 == 0) {
      start = (int)std::floor((x - 1.0) / 2.0) - (nI / 2 - 1);
    } else {
      int best = 0;
      for (int p = 1; p < N; ++p)
        if (std::fabs(2.0 * p + 1.0 - x) < std::fabs(2.0 * best + 1.0 - x)) best = p;
      start = best - nI / 2;
    }
    start = std::min(std::max(start, 0), N - nI);
    for (int m = 0; m < nI; ++m) {
      const double xm = 2.0 * (start + m) + 1.0;
      double w = 1.0;
      for (int q = 0; q < nI; ++q)
        if (q != m) {
          const double xq = 2.0 * (start + q) + 1.0;
          w *= (x - xq) / (xm - xq);
        }
      J[(size_t)j * N + start + m] = w;
    }
  }
  return J;
}

// Bump allocator that collects host arrays and uploads them in one copy.
struct Arena {
  std::vector<char> host;
  char* dev = nullptr;
  template <typename T>
  size_t add(const T* p, size_t n) {
    size_t off = (host.size() + 255) & ~(size_t)255;
    host.resize(off + n * sizeof(T));
    if (n) std::memcpy(host.data() + off, p, n * sizeof(T));
    return off;
  }
  template <typename T>
  size_t add(const std::vector<T>& v) { return add(v.data(), v.size()); }
  template <typename T>
  T* at(size_t off) const { return reinterpret_cast<T*>(dev + off); }
};

struct Inst {  // one FMM over one refinement level of one problem
  int p, l, variant;
  int top = 0;
  std::vector<std::vector<I3>> lv;                       // block coords per octree level
  std::vector<std::unordered_map<uint64_t, int>> idx;    // coords -> index per level
  std::vector<int> gid0;                                 // first global id per level
  std::vector<std::vector<uint8_t>> is_src, need_tgt;
  double h = 1.0;
};

struct LevelInfo {
  std::vector<I3> c;
  std::vector<uint8_t> leaf;
  std::vector<uint8_t> ext;  // non-leaf block or a neighbour of one: where W^l is needed
  std::vector<uint8_t> want; // the caller wants u here (flgf_blockset_create_masked; all by default)
  std::unordered_map<uint64_t, int> idx;
  int fw0 = 0;      // first block in fuser / fwork
  int ugid0 = 0;    // first global id of u^l (instance 0, octree level 0)
  int inst0 = -1, inst1 = -1;
  double h = 1.0;
  size_t nbr6_off = 0;  // arena offset of the face-neighbour table
};

struct Problem {
  int L = 1;
  double h0 = 1.0;
  std::vector<LevelInfo> lev;
};

struct PhaseOff {  // arena offsets and counts of one phase's launch lists
  int gid_begin = 0, nblocks = 0;
  int n_prep = 0; size_t prep_src = 0, prep_dst = 0, prep_zero = 0;
  std::vector<int> n_ant; std::vector<size_t> ant_par, ant_ch;
  int n_fwd = 0; size_t fwd_gid = 0, fwd_sid = 0;
  int n_groups_dense = 0, n_work = 0, max_units = 0;
  size_t hgroups = 0, work = 0, src_ids = 0, tgt_ids = 0, par_tab = 0;
  int n_groups = 0, max_group_src = 0; size_t groups = 0, l_tgt = 0, l_len = 0, l_ent = 0, l_src = 0;
  int n_fl = 0, fl_max_cells = 0, fl_max_parents = 0;
  size_t fl_groups = 0, fl_rows = 0, fl_dlms = 0, fl_tgt = 0, fl_cells = 0;
  int fl_ncomp = 1, fl_cstride = 0;  // components sharing the frequency-lane groups, their column stride
  bool fl_split = false;              // rows nearly all full: the two-path product form
  int n_fll = 0; size_t fll_groups = 0, fll_tgt = 0, fll_beg = 0, fll_len = 0, fll_ent = 0;
  int n_inv = 0, n_inv0 = 0; size_t inv_sid = 0, inv_gid = 0, inv_scale = 0;  // finest octree level first (n_inv0)
  std::vector<int> n_itp; std::vector<size_t> itp_ch, itp_par, itp_cpos;
  int n_sel = 0; size_t sel_src = 0, sel_dst = 0;
  int n_selw = 0; size_t selw_src = 0, selw_dst = 0;
  int n_acc = 0; size_t acc_nbr = 0, acc_fine = 0, acc_cpos = 0;
  int n_accw = 0; size_t accw_nbr = 0, accw_fine = 0, accw_cpos = 0;
  int n_cor = 0; size_t cor_nbr = 0, cor_fine = 0, cor_cpos = 0, cor_ih2 = 0;
  int n_crs = 0; size_t crs_coarse = 0, crs_fine = 0;  // coarsening of level l from l+1
};

}  // namespace

namespace {
struct AdjOff {  // adjoint lists of one phase (level), besides its FMM lists
  int n_prep = 0; size_t prep_dst = 0, prep_s1 = 0, prep_s2 = 0;   // nodes = gseed(masked) + gW(ext)
  int n_gacc = 0; size_t gacc_dst = 0, gacc_s1 = 0, gacc_s2 = 0;   // gf += A^T results
  int n_gtmp = 0; size_t gtmp_dst = 0, gtmp_s1 = 0, gtmp_s2 = 0;   // gtmp = gseed + gW(ext)
  int n_cf0 = 0; size_t cf0_nbr = 0, cf0_fine = 0, cf0_cpos = 0;   // gW^{l-1} += J^T gtmp
  int n_cf1 = 0; size_t cf1_nbr = 0, cf1_fine = 0, cf1_cpos = 0, cf1_ih2 = 0;  // gW^l += (L J)^T gf^{l+1}
};
}  // namespace

struct flgf_blockset {
  flgf_ctx* ctx = nullptr;
  std::vector<Problem> prob;
  std::vector<Inst> inst;
  std::vector<Inst> adj_inst;   // transposed leaf-only instances (sources: non-leaf + buffer, targets: leaf)
  std::vector<PhaseOff> ph;
  std::vector<PhaseOff> aph;    // FMM lists of the adjoint
  std::vector<AdjOff> adj;
  int Lmax = 0, G = 0, B = 0, max_phase_blocks = 0, max_level_blocks = 0;
  int64_t dof = 0, pairs = 0, n_fwd = 0, n_inv = 0, n_koff = 0;
  Arena ar;
  void* nodes = nullptr;
  void* unodes = nullptr;
  void* fuser = nullptr;
  void* fwork = nullptr;
  void* wfield = nullptr;  // leaf-source field W^l on non-leaf blocks and their buffer, [B][N^3]
  void* gseed = nullptr;   // adjoint of u (loaded by the caller), [B][N^3]
  void* gW = nullptr;      // adjoint of W, [B][N^3]
  void* gf = nullptr;      // adjoint of the level sources -> the gradient, [B][N^3]
  void* gtmp = nullptr;    // [B][N^3]
  void* aunodes = nullptr; // FMM outputs of the adjoint, [G][N^3] (the potentials stay in unodes)
  bool adj_solved = false;
  void* spec = nullptr;
  void* acc = nullptr;
  void* lap_in = nullptr;
  void* lap_out = nullptr;
  int* d_err = nullptr;
  // host source loads run on their own stream: they wait only until the
  // solve in flight has copied the source buffer (ev_fuser_free), so they
  // overlap the rest of that solve; the next solve waits for ev_loaded
  cudaStream_t cstream = nullptr;
  // adjoint lists and buffers, built on first use (flgf_load_adjoint / flgf_solve_adjoint)
  Arena aar;
  bool adj_ready = false;
  cudaEvent_t ev_fuser_free = nullptr, ev_loaded = nullptr, ev_dev_load = nullptr;
  bool load_pending = false;
  bool correction = true, solved = false;
  bool use_graph = false, timing = false;
  bool compensated = false;  // FLGF_OPT_COMPENSATED (FP32 block sets)
  bool masked = false;       // created with a target mask (flgf_blockset_create_masked)
  int ncomp = 1;             // components of a vector block set (flgf_blockset_create_vector)
  cudaGraphExec_t gexec = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;  // (stage, (start, end))
  size_t ev_used = 0;
  double stage_ms[7] = {0, 0, 0, 0, 0, 0, 0};
  int timed_solves = 0;
  bool ev_pending = false;
  int64_t launches = 0;  // kernels enqueued by the last solve
  bool capturing = false;
};

// ----------------------------------------------------------------------------
// Context
// ----------------------------------------------------------------------------
extern "C" void flgf_default_opts(flgf_opts* o) {
  if (!o) return;
  o->N = 16;
  o->n_interp = 6;
  o->precision = FLGF_FP64;
  o->max_oct_levels = 6;
  o->table_radius = 100;
  o->asym_radius = 600;
  o->stream = nullptr;
}

extern "C" const char* flgf_last_error(const flgf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" void flgf_destroy(flgf_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->d_table);
  cudaFree(ctx->d_J1);
  cudaFree(ctx->d_kspec);
  delete ctx;
}

extern "C" int flgf_create(flgf_ctx** out, const flgf_opts* o) {
  if (!out || !o) return FLGF_EINVAL;
  *out = nullptr;
  flgf_ctx* ctx = new (std::nothrow) flgf_ctx();
  if (!ctx) return FLGF_ENOMEM;
  auto bad = [&](const std::string& m) { delete ctx; (void)m; return FLGF_EINVAL; };
  if (o->N != 8 && o->N != 16) return bad("N must be 8 or 16");
  if (o->n_interp < 2 || o->n_interp > std::min(o->N, 10)) return bad("n_interp out of range");
  if (o->precision != FLGF_FP64 && o->precision != FLGF_FP32) return bad("precision");
  if (o->max_oct_levels < 1 || o->max_oct_levels > 8) return bad("max_oct_levels");
  if (o->table_radius < 1 || o->table_radius > 200 || o->asym_radius < o->table_radius) return bad("radii");
  ctx->N = o->N;
  ctx->nI = o->n_interp;
  ctx->prec = o->precision;
  ctx->max_oct = o->max_oct_levels;
  ctx->R = o->table_radius;
  ctx->RA = o->asym_radius;
  ctx->stream = (cudaStream_t)o->stream;
  ctx->J1 = lagrange_matrix(ctx->N, ctx->nI);
  const int N = ctx->N, P = 2 * N, NW = nfreq(N);
  const int R = ctx->R;
  double* B = nullptr;
  double* karr = nullptr;
  double* tmp = nullptr;
  auto cleanup = [&]() { cudaFree(B); cudaFree(karr); cudaFree(tmp); };
  auto ck = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return FLGF_OK;
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return FLGF_ECUDA;
  };
  int rc;
#define STEP(call)                          \
  if ((rc = ck((call), #call)) != FLGF_OK) { \
    cleanup();                              \
    flgf_destroy(ctx);                      \
    return rc;                              \
  }
  STEP(fft_init_constants());
  STEP(cudaMalloc(&ctx->d_J1, sizeof(double) * ctx->J1.size()));
  STEP(cudaMemcpy(ctx->d_J1, ctx->J1.data(), sizeof(double) * ctx->J1.size(), cudaMemcpyHostToDevice));
  const size_t nq = (size_t)quad_nodes();
  STEP(cudaMalloc(&B, sizeof(double) * (R + 2) * nq));
  STEP(cudaMalloc(&ctx->d_table, sizeof(double) * (size_t)(R + 1) * (R + 1) * (R + 1)));
  STEP(cudaMemsetAsync(ctx->d_table, 0, sizeof(double) * (size_t)(R + 1) * (R + 1) * (R + 1), ctx->stream));
  STEP(launch_bessel_table(B, R, ctx->stream));
  STEP(launch_lgf_table(B, R, ctx->d_table, R, ctx->stream));
  const size_t csz = ctx->prec == FLGF_FP64 ? 16 : 8;
  ctx->kstride = (size_t)kNOff * NW;
  STEP(cudaMalloc(&ctx->d_kspec, csz * ctx->kstride * ctx->max_oct));
  STEP(cudaMalloc(&karr, sizeof(double) * (size_t)kNOff * P * P * P));
  STEP(cudaMalloc(&tmp, 2 * 16 * (size_t)kNOff * NW));
  for (int k = 0; k < ctx->max_oct; ++k) {
    STEP(launch_kernel_arrays(ctx->d_table, R, (double)R, (double)ctx->RA, N, k, karr, ctx->stream));
    void* lvl = (char*)ctx->d_kspec + csz * ctx->kstride * k;
    if (ctx->prec == FLGF_FP64) {
      STEP(launch_kernel_spectra<double>(N, karr, lvl, tmp, k >= 1 ? 1 : 0, ctx->stream));
    } else {
      STEP(launch_kernel_spectra<float>(N, karr, lvl, tmp, k >= 1 ? 1 : 0, ctx->stream));
    }
  }
  STEP(cudaStreamSynchronize(ctx->stream));
#undef STEP
  cleanup();
  *out = ctx;
  return FLGF_OK;
}

extern "C" int flgf_lgf_eval(flgf_ctx* ctx, int n, const int32_t* pts, double* out) {
  if (!ctx || n < 0 || (n > 0 && (!pts || !out))) return fail(ctx, FLGF_EINVAL, "lgf_eval: bad arguments");
  if (n == 0) return FLGF_OK;
  int32_t* dp = nullptr;
  double* dv = nullptr;
  CK(cudaMalloc(&dp, sizeof(int32_t) * 3 * n));
  cudaError_t e = cudaMalloc(&dv, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, pts, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_lgf_eval(ctx->d_table, ctx->R, (double)ctx->R, (double)ctx->RA, dp, n, dv, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dv, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dp);
  cudaFree(dv);
  if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("lgf_eval: ") + cudaGetErrorString(e));
  return FLGF_OK;
}

extern "C" int flgf_kernel_spectrum(flgf_ctx* ctx, int k, int d0, int d1, int d2, double* out) {
  if (!ctx || !out || k < 0 || k >= ctx->max_oct || std::abs(d0) > 3 || std::abs(d1) > 3 || std::abs(d2) > 3)
    return fail(ctx, FLGF_EINVAL, "kernel_spectrum: bad arguments");
  const int N = ctx->N, NW = nfreq(N);
  const int d = off_index(d0, d1, d2);
  const bool f64 = ctx->prec == FLGF_FP64;
  const int T = f64 ? 2 : 4;
  const size_t csz = f64 ? 16 : 8;
  std::vector<char> lvl(csz * ctx->kstride);
  CK(cudaMemcpyAsync(lvl.data(), (char*)ctx->d_kspec + csz * ctx->kstride * k, lvl.size(), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int w = 0; w < NW; ++w) {
    const size_t ix = ((size_t)(w / T) * kNOff + d) * T + (w % T);
    if (f64) {
      const double* v = reinterpret_cast<const double*>(lvl.data()) + 2 * ix;
      out[2 * w] = v[0];
      out[2 * w + 1] = v[1];
    } else {
      const float* v = reinterpret_cast<const float*>(lvl.data()) + 2 * ix;
      out[2 * w] = v[0];
      out[2 * w + 1] = v[1];
    }
  }
  return FLGF_OK;
}

// ----------------------------------------------------------------------------
// Block set compilation
// ----------------------------------------------------------------------------
namespace {

int build_octree(Inst& in, const std::vector<I3>& base, int max_oct, std::string& err) {
  in.lv.clear();
  in.lv.push_back(base);
  int k = 0;
  while (true) {
    I3 lo = {INT32_MAX, INT32_MAX, INT32_MAX}, hi = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (const auto& c : in.lv[k])
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], c[a] >> 1);
        hi[a] = std::max(hi[a], c[a] >> 1);
      }
    if (hi[0] - lo[0] <= 1 && hi[1] - lo[1] <= 1 && hi[2] - lo[2] <= 1) break;
    std::vector<I3> par;
    par.reserve(in.lv[k].size());
    for (const auto& c : in.lv[k]) par.push_back({c[0] >> 1, c[1] >> 1, c[2] >> 1});
    std::sort(par.begin(), par.end());
    par.erase(std::unique(par.begin(), par.end()), par.end());
    in.lv.push_back(par);
    ++k;
  }
  in.top = k;
  if (in.top + 1 > max_oct) {
    err = "block set needs " + std::to_string(in.top + 1) + " octree levels; context caches " +
          std::to_string(max_oct) + " (raise max_oct_levels)";
    return FLGF_EINVAL;
  }
  in.idx.assign(in.lv.size(), {});
  for (size_t q = 0; q < in.lv.size(); ++q)
    for (size_t i = 0; i < in.lv[q].size(); ++i) in.idx[q][key3(in.lv[q][i])] = (int)i;
  return FLGF_OK;
}

}  // namespace

extern "C" void flgf_blockset_destroy(flgf_blockset* bs) {
  if (!bs) return;
  if (bs->gexec) cudaGraphExecDestroy(bs->gexec);
  for (auto& e : bs->ev) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  cudaFree(bs->ar.dev);
  cudaFree(bs->nodes);
  cudaFree(bs->unodes);
  cudaFree(bs->fuser);
  cudaFree(bs->fwork);
  cudaFree(bs->wfield);
  cudaFree(bs->gseed);
  cudaFree(bs->gW);
  cudaFree(bs->gf);
  cudaFree(bs->gtmp);
  cudaFree(bs->aunodes);
  cudaFree(bs->spec);
  cudaFree(bs->acc);
  cudaFree(bs->lap_in);
  cudaFree(bs->lap_out);
  cudaFree(bs->d_err);
  if (bs->ev_fuser_free) cudaEventDestroy(bs->ev_fuser_free);
  if (bs->ev_loaded) cudaEventDestroy(bs->ev_loaded);
  if (bs->ev_dev_load) cudaEventDestroy(bs->ev_dev_load);
  if (bs->cstream) cudaStreamDestroy(bs->cstream);
  cudaFree(bs->aar.dev);
  delete bs;
}

// FMM launch lists of phase l for the given instances (their is_src /
// need_tgt masks select sources and targets), appended to arena ar.
static void build_fmm(flgf_blockset* bs, Arena& ar, int l, const std::vector<const Inst*>& insts, PhaseOff& ph, bool count,
                      int ncomp) {
  flgf_ctx* ctx = bs->ctx;
  const int N = ctx->N;
  const int TP[3] = {ctx->tile[0], ctx->tile[1], ctx->tile[2]};  // tile in parents (<= 128: 256 threads)
  std::vector<int> prep_src, prep_dst;
  std::vector<uint8_t> prep_zero;
  int maxtop = 0;
  for (const Inst* in : insts) maxtop = std::max(maxtop, in->top);
  std::vector<std::vector<int>> ant_par(maxtop + 1), ant_ch(maxtop + 1);
  std::vector<std::vector<int>> itp_ch(maxtop + 1), itp_par(maxtop + 1), itp_cpos(maxtop + 1);
  // inverse FFT list: finest octree level, then the coarser ones (their own launch)
  std::vector<int> fwd_gid, fwd_sid, inv_sid, inv_gid, inv_sid_c, inv_gid_c;
  std::vector<double> inv_scale, inv_scale_c;
  // parents with targets of dense tiles per octree level, in tile order
  std::vector<std::vector<ParentRec>> dpool;
  std::vector<ListGroup> groups;
  std::vector<int> l_tgt, l_len, l_ent, l_src;
  int max_group_src = 0;
  // targets of sparse tiles per octree level, in tile order: (target id, pair list)
  std::vector<std::vector<std::pair<int, std::vector<int>>>> lpool;
  const int nchunk = ctx->prec == FLGF_FP64 ? nchunks<double>(N) : nchunks<float>(N);
  // FP32 frequency-lane MAC: the dense tiles' parents go to its groups (sparse
  // tiles still to the pair lists)
  const bool fl = ctx->prec == FLGF_FP32 && ctx->mac >= 1;
  // FP32 pair lists of sparse tiles in frequency lanes (mac 1) or in the
  // shared-memory pair-list kernel (mac 0 and 2)
  const bool fll_lists = ctx->prec == FLGF_FP32 && ctx->mac == 1;
  // vector block set (identical meshes, problem c = component c): component
  // 0's dense tiles serve every component (columns + c * cstride) in the same
  // CTAs, which stage the kernel spectra and group tables once
  const int vcomp = fl ? ncomp : 1;
  const int list_pct = ctx->list_pct;
  // interaction tiles of one (instance, octree level): the expensive part of
  // list building, run on the host's cores (see below)
  struct TileJob {
    const Inst* inp;
    int k;
    std::vector<ParentRec> drecs;                           // parents of dense tiles, in tile order
    std::vector<std::pair<int, std::vector<int>>> lrecs;   // targets of sparse tiles with their pair lists
    int64_t pairs = 0;
  };
  std::vector<TileJob> jobs;
  auto run_tiles = [&](TileJob& job) {
    const Inst& in = *job.inp;
    const size_t k = (size_t)job.k;
    // interaction tiles of this octree level
    I3 lo = {INT32_MAX, INT32_MAX, INT32_MAX}, hi = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (const auto& c : in.lv[k])
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], c[a] >> 1);
        hi[a] = std::max(hi[a], c[a] >> 1);
      }
    // block index by coordinates: a dense grid over the level's box when it is
    // small enough (every lookup below stays inside [2 lo, 2 hi + 1]), else the hash map
    const I3 glo = {2 * lo[0], 2 * lo[1], 2 * lo[2]};
    const int64_t gd[3] = {2 * (int64_t)(hi[0] - lo[0]) + 2, 2 * (int64_t)(hi[1] - lo[1]) + 2,
                           2 * (int64_t)(hi[2] - lo[2]) + 2};
    const bool use_grid = gd[0] * gd[1] * gd[2] <= ((int64_t)1 << 24);
    std::vector<int> grid;
    if (use_grid) {
      grid.assign((size_t)(gd[0] * gd[1] * gd[2]), -1);
      for (size_t i = 0; i < in.lv[k].size(); ++i) {
        const I3& c = in.lv[k][i];
        grid[((size_t)(c[0] - glo[0]) * gd[1] + (c[1] - glo[1])) * gd[2] + (c[2] - glo[2])] = (int)i;
      }
    }
    auto lookup = [&](int a, int b, int c2) -> int {
      if (use_grid) {
        const int64_t x = a - glo[0], y = b - glo[1], z = c2 - glo[2];
        if (x < 0 || y < 0 || z < 0 || x >= gd[0] || y >= gd[1] || z >= gd[2]) return -1;
        return grid[((size_t)x * gd[1] + y) * gd[2] + z];
      }
      auto it = in.idx[k].find(key3(a, b, c2));
      return it == in.idx[k].end() ? -1 : it->second;
    };
    const bool excl = k > 0;
    for (int t0 = lo[0]; t0 <= hi[0]; t0 += TP[0])
      for (int t1 = lo[1]; t1 <= hi[1]; t1 += TP[1])
        for (int t2 = lo[2]; t2 <= hi[2]; t2 += TP[2]) {
          struct { int P[3], r0[3], Rg[3]; } tl;  // tile and its region (tile + 1 parent, clipped)
          const int t[3] = {t0, t1, t2};
          for (int a = 0; a < 3; ++a) {
            tl.P[a] = std::min(TP[a], hi[a] - t[a] + 1);
            tl.r0[a] = std::max(t[a] - 1, lo[a]);
            tl.Rg[a] = std::min(t[a] + tl.P[a], hi[a]) - tl.r0[a] + 1;
          }
          std::vector<int> tg;
          bool any = false;
          for (int x = 0; x < 2 * tl.P[0]; ++x)
            for (int y = 0; y < 2 * tl.P[1]; ++y)
              for (int z = 0; z < 2 * tl.P[2]; ++z) {
                const int i = lookup(2 * t0 + x, 2 * t1 + y, 2 * t2 + z);
                const bool need = i >= 0 && in.need_tgt[k][i];
                tg.push_back(need ? in.gid0[k] + i - ph.gid_begin : -1);
                any |= need;
              }
          if (!any) continue;
          // source slots in parity-major order: slot = b * NQ + q
          const int NQ = tl.Rg[0] * tl.Rg[1] * tl.Rg[2];
          std::vector<int> sg(8 * NQ, -1);
          for (int x = 0; x < 2 * tl.Rg[0]; ++x)
            for (int y = 0; y < 2 * tl.Rg[1]; ++y)
              for (int z = 0; z < 2 * tl.Rg[2]; ++z) {
                const int i = lookup(2 * tl.r0[0] + x, 2 * tl.r0[1] + y, 2 * tl.r0[2] + z);
                const int b = ((x & 1) << 2) | ((y & 1) << 1) | (z & 1);
                const int qq = ((x >> 1) * tl.Rg[1] + (y >> 1)) * tl.Rg[2] + (z >> 1);
                sg[b * NQ + qq] = i >= 0 && in.is_src[k][i] ? in.gid0[k] + i - ph.gid_begin : -1;
              }
          // the interacting (target, source) pairs of every target: the
          // candidates are the children of its parent's 27 neighbours
          std::vector<std::vector<int>> plist(tg.size());  // (source id << 9) | offset index
          int64_t useful = 0;
          for (int x = 0; x < 2 * tl.P[0]; ++x)
            for (int y = 0; y < 2 * tl.P[1]; ++y)
              for (int z = 0; z < 2 * tl.P[2]; ++z) {
                const int ti = (x * 2 * tl.P[1] + y) * 2 * tl.P[2] + z;
                if (tg[ti] < 0) continue;
                const int tc[3] = {2 * t0 + x, 2 * t1 + y, 2 * t2 + z};
                for (int e = 0; e < 27; ++e)
                  for (int b = 0; b < 8; ++b) {
                    const int sc[3] = {2 * ((tc[0] >> 1) + e / 9 - 1) + (b >> 2),
                                       2 * ((tc[1] >> 1) + (e / 3) % 3 - 1) + ((b >> 1) & 1),
                                       2 * ((tc[2] >> 1) + e % 3 - 1) + (b & 1)};
                    int rr[3];
                    bool in = true, near = true;
                    for (int a = 0; a < 3; ++a) {
                      rr[a] = sc[a] - 2 * tl.r0[a];
                      in &= rr[a] >= 0 && rr[a] < 2 * tl.Rg[a];
                      near &= std::abs(sc[a] - tc[a]) <= 1;
                    }
                    if (!in || (excl && near)) continue;
                    const int bb = ((rr[0] & 1) << 2) | ((rr[1] & 1) << 1) | (rr[2] & 1);
                    const int qq = ((rr[0] >> 1) * tl.Rg[1] + (rr[1] >> 1)) * tl.Rg[2] + (rr[2] >> 1);
                    const int sid = sg[bb * NQ + qq];
                    if (sid < 0) continue;
                    plist[ti].push_back((sid << 9) | off_index(tc[0] - sc[0], tc[1] - sc[1], tc[2] - sc[2]));
                  }
                useful += (int64_t)plist[ti].size();
              }
          job.pairs += useful;
          // parent records of the tile's parents that have targets
          std::vector<ParentRec> recs;
          int64_t dense = 0;  // complex MACs per frequency of the parent-group kernel
          for (int p0 = 0; p0 < tl.P[0]; ++p0)
            for (int p1 = 0; p1 < tl.P[1]; ++p1)
              for (int p2 = 0; p2 < tl.P[2]; ++p2) {
                ParentRec r;
                bool has = false;
                for (int a = 0; a < 8; ++a) {
                  r.tgt[a] = tg[((2 * p0 + (a >> 2)) * 2 * tl.P[1] + 2 * p1 + ((a >> 1) & 1)) * 2 * tl.P[2] + 2 * p2 +
                                (a & 1)];
                  has |= r.tgt[a] >= 0;
                }
                if (!has) continue;
                const int pc[3] = {t0 + p0, t1 + p1, t2 + p2};
                for (int e = 0; e < 27; ++e) {
                  const int ee[3] = {e / 9 - 1, (e / 3) % 3 - 1, e % 3 - 1};
                  int q[3];
                  bool inr = !(excl && e == 13);
                  for (int a = 0; a < 3; ++a) {
                    q[a] = pc[a] + ee[a] - tl.r0[a];
                    inr &= q[a] >= 0 && q[a] < tl.Rg[a];
                  }
                  bool any_src = false;
                  for (int b = 0; b < 8; ++b) {
                    r.cell[e][b] = inr ? sg[b * NQ + (q[0] * tl.Rg[1] + q[1]) * tl.Rg[2] + q[2]] : -1;
                    any_src |= r.cell[e][b] >= 0;
                  }
                  dense += any_src ? 64 : 0;
                }
                recs.push_back(r);
              }
          if (useful * 100 < (int64_t)list_pct * dense) {
            // sparse tile: its targets join the pair-list pool of octree level k
            for (int ti = 0; ti < (int)tg.size(); ++ti)
              if (tg[ti] >= 0) job.lrecs.push_back({tg[ti], std::move(plist[ti])});
            continue;
          }
          job.drecs.insert(job.drecs.end(), recs.begin(), recs.end());
        }
  };
  for (const Inst* inp : insts) {
    const Inst& in = *inp;
    const LevelInfo& L = bs->prob[in.p].lev[l];
    for (size_t b = 0; b < L.c.size(); ++b) {
      prep_src.push_back(L.fw0 + (int)b);
      prep_dst.push_back(in.gid0[0] + (int)b);
      prep_zero.push_back(in.variant == 1 && !L.leaf[b]);
    }
    for (int k = 1; k <= in.top; ++k) {
      for (size_t i = 0; i < in.lv[k].size(); ++i) {
        const I3& c = in.lv[k][i];
        ant_par[k].push_back(in.gid0[k] + (int)i);
        for (int a = 0; a < 8; ++a) {
          const I3 ch = {2 * c[0] + (a >> 2), 2 * c[1] + ((a >> 1) & 1), 2 * c[2] + (a & 1)};
          auto it = in.idx[k - 1].find(key3(ch));
          ant_ch[k].push_back(it == in.idx[k - 1].end() ? -1 : in.gid0[k - 1] + it->second);
        }
      }
    }
    for (size_t k = 0; k < in.lv.size(); ++k) {
      for (size_t i = 0; i < in.lv[k].size(); ++i) {
        const int gid = in.gid0[k] + (int)i;
        if (in.is_src[k][i]) {
          fwd_gid.push_back(gid);
          fwd_sid.push_back(gid - ph.gid_begin);
        }
        if (in.need_tgt[k][i]) {
          (k == 0 ? inv_sid : inv_sid_c).push_back(gid - ph.gid_begin);
          (k == 0 ? inv_gid : inv_gid_c).push_back(gid);
          (k == 0 ? inv_scale : inv_scale_c).push_back(in.h * in.h);
          if ((int)k < in.top) {
            const I3& c = in.lv[k][i];
            const int pi = in.idx[k + 1].at(key3(c[0] >> 1, c[1] >> 1, c[2] >> 1));
            itp_ch[k].push_back(gid);
            itp_par[k].push_back(in.gid0[k + 1] + pi);
            itp_cpos[k].push_back(((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1));
          }
        }
      }
      jobs.push_back(TileJob{&in, (int)k});
    }
  }
  const int n_inv0 = (int)inv_gid.size();
  inv_gid.insert(inv_gid.end(), inv_gid_c.begin(), inv_gid_c.end());
  inv_sid.insert(inv_sid.end(), inv_sid_c.begin(), inv_sid_c.end());
  inv_scale.insert(inv_scale.end(), inv_scale_c.begin(), inv_scale_c.end());
  // run the tile jobs on the host's cores; the results are merged in job order,
  // so the launch lists do not depend on the number of threads
  {
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nth = std::min<size_t>(jobs.size(), std::max(1u, std::min(hw, 32u)));
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      for (size_t j = next++; j < jobs.size(); j = next++) run_tiles(jobs[j]);
    };
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nth; ++t) {
      try {
        pool.emplace_back(worker);
      } catch (...) {  // no more threads: the workers already started and this one finish the jobs
        break;
      }
    }
    worker();
    for (auto& th : pool) th.join();
  }
  for (TileJob& job : jobs) {
    if (count) bs->pairs += job.pairs;
    if (vcomp > 1 && job.inp->p > 0) job.drecs.clear();  // component 0's groups serve it
    if (!job.drecs.empty()) {
      if ((int)dpool.size() <= job.k) dpool.resize(job.k + 1);
      dpool[job.k].insert(dpool[job.k].end(), job.drecs.begin(), job.drecs.end());
    }
    if (!job.lrecs.empty()) {
      if ((int)lpool.size() <= job.k) lpool.resize(job.k + 1);
      for (auto& r : job.lrecs) lpool[job.k].push_back(std::move(r));
    }
  }
  // dense MAC: parent groups of every octree level (or frequency-lane groups)
  HadLists hl;
  FlLists fll;
  for (int k = 0; k < (int)dpool.size(); ++k) {
    if (fl)
      pack_fl_groups(k, dpool[k], fll);
    else
      pack_parent_groups(k, dpool[k], nchunk, had_kernel_units(ctx->prec == FLGF_FP64), hl, ctx->order_by_list);
  }
  ph.n_fl = (int)fll.groups.size();
  {
    size_t rows = 0, full = 0;
    for (const FlGroup& g : fll.groups)
      for (int m = 0; m < g.nact; ++m) {
        const int n = fll.rows[(size_t)(g.row_off + m) * kFlRowStride];
        rows += n;
        for (int j = 0; j < n; ++j) full += fll.dlms[(size_t)(g.row_off + m) * kFlDelta + j] >> 31;
      }
    ph.fl_split = rows > 0 && (double)full >= kFlSplitFullFraction * (double)rows;
  }
  ph.fl_ncomp = vcomp;
  ph.fl_cstride = ph.nblocks / vcomp;
  ph.fl_max_cells = fll.max_cells;
  ph.fl_max_parents = fll.max_parents;
  ph.fl_groups = ar.add(fll.groups);
  ph.fl_rows = ar.add(fll.rows);
  ph.fl_dlms = ar.add(fll.dlms);
  ph.fl_tgt = ar.add(fll.tgt_ids);
  ph.fl_cells = ar.add(fll.cells);
  FllLists fq;
  if (fll_lists) {
    for (int k = 0; k < (int)lpool.size(); ++k) pack_fll_groups(k, lpool[k], fq);
    lpool.clear();
  }
  ph.n_fll = (int)fq.groups.size();
  ph.fll_groups = ar.add(fq.groups);
  ph.fll_tgt = ar.add(fq.tgt);
  ph.fll_beg = ar.add(fq.beg);
  ph.fll_len = ar.add(fq.len);
  ph.fll_ent = ar.add(fq.ent);
  // pair-list groups: consecutive pool targets (spatially close, so their
  // source sets overlap) up to kListTargets targets or kListMaxSrc sources
  for (int k = 0; k < (int)lpool.size(); ++k) {
    const auto& pool = lpool[k];
    size_t pos = 0;
    while (pos < pool.size()) {
      std::unordered_map<int, int> slot;
      std::vector<int> gsrc, members;
      while (pos < pool.size() && (int)members.size() < kListTargets) {
        const auto& pl = pool[pos].second;
        int add = 0;
        for (int w : pl) add += slot.count(w >> 9) ? 0 : 1;
        if (!members.empty() && (int)gsrc.size() + add > kListMaxSrc) break;
        for (int w : pl)
          if (!slot.count(w >> 9)) {
            slot.emplace(w >> 9, (int)gsrc.size());
            gsrc.push_back(w >> 9);
          }
        members.push_back((int)pos++);
      }
      // longest lists first: the threads of a warp run similar trip counts
      std::stable_sort(members.begin(), members.end(),
                       [&](int a, int b) { return pool[a].second.size() > pool[b].second.size(); });
      ListGroup g;
      g.level = k;
      g.ntgt = (int)members.size();
      g.maxlen = (int)pool[members[0]].second.size();
      g.tgt_off = (int)l_tgt.size();
      g.len_off = (int)l_len.size();
      g.ent_off = (int)l_ent.size();
      g.src_off = (int)l_src.size();
      g.nsrc = (int)gsrc.size();
      l_ent.resize(l_ent.size() + (size_t)g.maxlen * kListTargets, 0);
      for (int m = 0; m < g.ntgt; ++m) {
        const auto& pl = pool[members[m]].second;
        l_tgt.push_back(pool[members[m]].first);
        l_len.push_back((int)pl.size());
        for (size_t j = 0; j < pl.size(); ++j)
          l_ent[g.ent_off + j * kListTargets + m] = (slot.at(pl[j] >> 9) << 9) | (pl[j] & 511);
      }
      l_src.insert(l_src.end(), gsrc.begin(), gsrc.end());
      max_group_src = std::max(max_group_src, g.nsrc);
      groups.push_back(g);
    }
  }
  if (count) {
    bs->n_fwd += (int64_t)fwd_gid.size();
    bs->n_inv += (int64_t)inv_gid.size();
    for (int k = 0; k <= maxtop; ++k) bs->n_koff += kNOff;
  }
  ph.n_prep = (int)prep_src.size();
  ph.prep_src = ar.add(prep_src);
  ph.prep_dst = ar.add(prep_dst);
  ph.prep_zero = ar.add(prep_zero);
  ph.n_ant.assign(maxtop + 1, 0);
  ph.ant_par.assign(maxtop + 1, 0);
  ph.ant_ch.assign(maxtop + 1, 0);
  ph.n_itp.assign(maxtop + 1, 0);
  ph.itp_ch.assign(maxtop + 1, 0);
  ph.itp_par.assign(maxtop + 1, 0);
  ph.itp_cpos.assign(maxtop + 1, 0);
  for (int k = 0; k <= maxtop; ++k) {
    // interpolation children grouped by child position: the CTAs resident on
    // an SM then take the same one of the kernel's per-axis code paths, which
    // keeps its instruction working set small (children are independent)
    {
      std::vector<int> ord(itp_ch[k].size());
      for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return itp_cpos[k][x] < itp_cpos[k][y]; });
      std::vector<int> ch(ord.size()), par(ord.size()), cp(ord.size());
      for (size_t i = 0; i < ord.size(); ++i) {
        ch[i] = itp_ch[k][ord[i]];
        par[i] = itp_par[k][ord[i]];
        cp[i] = itp_cpos[k][ord[i]];
      }
      itp_ch[k].swap(ch);
      itp_par[k].swap(par);
      itp_cpos[k].swap(cp);
    }
    ph.n_ant[k] = (int)ant_par[k].size();
    ph.ant_par[k] = ar.add(ant_par[k]);
    ph.ant_ch[k] = ar.add(ant_ch[k]);
    ph.n_itp[k] = (int)itp_ch[k].size();
    ph.itp_ch[k] = ar.add(itp_ch[k]);
    ph.itp_par[k] = ar.add(itp_par[k]);
    ph.itp_cpos[k] = ar.add(itp_cpos[k]);
  }
  ph.n_fwd = (int)fwd_gid.size();
  ph.fwd_gid = ar.add(fwd_gid);
  ph.fwd_sid = ar.add(fwd_sid);
  ph.n_groups_dense = (int)hl.groups.size();
  ph.hgroups = ar.add(hl.groups);
  ph.max_units = hl.max_units;
  std::vector<HadWork>& work = hl.work;
  // chunk-major order: the groups sharing a frequency chunk run back to back,
  // so the chunk's kernel spectra and the shared halo spectra stay in L2
  std::stable_sort(work.begin(), work.end(), [](const HadWork& x, const HadWork& y) { return x.chunk0 < y.chunk0; });
  ph.n_work = (int)work.size();
  ph.work = ar.add(work);
  ph.src_ids = ar.add(hl.src_ids);
  ph.tgt_ids = ar.add(hl.tgt_ids);
  ph.par_tab = ar.add(hl.par_tab);
  ph.n_groups = (int)groups.size();
  ph.max_group_src = max_group_src;
  ph.groups = ar.add(groups);
  ph.l_tgt = ar.add(l_tgt);
  ph.l_len = ar.add(l_len);
  ph.l_ent = ar.add(l_ent);
  ph.l_src = ar.add(l_src);
  ph.n_inv = (int)inv_gid.size();
  ph.n_inv0 = n_inv0;
  ph.inv_sid = ar.add(inv_sid);
  ph.inv_gid = ar.add(inv_gid);
  ph.inv_scale = ar.add(inv_scale);
}

// Mesh checks, octrees and launch lists of a block set: host work only (no
// CUDA call), so the planning can be exercised without a GPU.  On failure the
// caller destroys bs.
static int plan_blockset(flgf_ctx* ctx, flgf_blockset* bs, int n_problems, const int* n_levels, const int* nblk,
                         const int32_t* coords, const double* h0, const uint8_t* want = nullptr) {
  const int N = ctx->N;
  const size_t N3 = (size_t)N * N * N;
  auto bail = [&](int code, const std::string& m) { return fail(ctx, code, m); };
  // ---- read and validate the mesh ------------------------------------------
  int q = 0;
  size_t ci = 0;
  bs->prob.resize(n_problems);
  for (int p = 0; p < n_problems; ++p) {
    Problem& P = bs->prob[p];
    P.L = n_levels[p];
    P.h0 = h0[p];
    if (P.L < 1 || P.L > 16) return bail(FLGF_EINVAL, "n_levels out of range");
    if (!(P.h0 > 0.0)) return bail(FLGF_EINVAL, "h0 must be positive");
    P.lev.resize(P.L);
    for (int l = 0; l < P.L; ++l, ++q) {
      LevelInfo& L = P.lev[l];
      const int nb = nblk[q];
      if (nb < 1) return bail(FLGF_EINVAL, "every level needs at least one block");
      L.c.resize(nb);
      L.want.assign(nb, 1);
      for (int b = 0; b < nb; ++b, ++ci) {
        if (want) L.want[b] = want[ci] != 0;
        for (int a = 0; a < 3; ++a) {
          const int v = coords[3 * ci + a];
          if (v < -(1 << 19) || v >= (1 << 19)) return bail(FLGF_EINVAL, "block coordinate out of range");
          L.c[b][a] = v;
        }
        if (!L.idx.emplace(key3(L.c[b]), b).second)
          return bail(FLGF_EMESH, "duplicate block in problem " + std::to_string(p) + " level " + std::to_string(l));
      }
      L.h = P.h0 / (double)(1 << l);
      bs->max_level_blocks = std::max(bs->max_level_blocks, nb);
    }
    for (int l = 0; l < P.L; ++l) {
      LevelInfo& L = P.lev[l];
      L.leaf.assign(L.c.size(), 1);
      if (l + 1 < P.L) {
        const LevelInfo& F = P.lev[l + 1];
        std::vector<int> nkids(L.c.size(), 0);
        for (const auto& c : F.c) {
          auto it = L.idx.find(key3(c[0] >> 1, c[1] >> 1, c[2] >> 1));
          if (it == L.idx.end())
            return bail(FLGF_EMESH, "level " + std::to_string(l + 1) + " block without a parent (problem " +
                                        std::to_string(p) + ")");
          nkids[it->second]++;
        }
        for (size_t b = 0; b < L.c.size(); ++b) {
          if (nkids[b] != 0 && nkids[b] != 8)
            return bail(FLGF_EMESH, "partially refined block (problem " + std::to_string(p) + ", level " +
                                        std::to_string(l) + ")");
          L.leaf[b] = nkids[b] == 0;
        }
        for (size_t b = 0; b < L.c.size(); ++b) {
          if (L.leaf[b]) continue;
          for (int e = 0; e < 27; ++e) {
            if (e == 13) continue;
            const I3 nbc = {L.c[b][0] + e / 9 - 1, L.c[b][1] + (e / 3) % 3 - 1, L.c[b][2] + e % 3 - 1};
            if (!L.idx.count(key3(nbc)))
              return bail(FLGF_EMESH, "refined block lacks its 26-neighbour buffer (problem " + std::to_string(p) +
                                          ", level " + std::to_string(l) + ")");
          }
        }
      }
      for (size_t b = 0; b < L.c.size(); ++b) bs->dof += L.leaf[b] ? (int64_t)N3 : 0;
      L.ext.assign(L.c.size(), 0);
      for (size_t b = 0; b < L.c.size(); ++b) {
        if (L.leaf[b]) continue;
        for (int e = 0; e < 27; ++e) {
          auto it = L.idx.find(key3(L.c[b][0] + e / 9 - 1, L.c[b][1] + (e / 3) % 3 - 1, L.c[b][2] + e % 3 - 1));
          if (it != L.idx.end()) L.ext[it->second] = 1;
        }
      }
    }
    bs->Lmax = std::max(bs->Lmax, P.L);
  }
  // ---- level storage -------------------------------------------------------
  for (auto& P : bs->prob)
    for (auto& L : P.lev) {
      L.fw0 = bs->B;
      bs->B += (int)L.c.size();
    }
  // ---- instances and global ids, phase by phase ----------------------------
  bs->ph.resize(bs->Lmax);
  std::string err;
  for (int l = 0; l < bs->Lmax; ++l) {
    PhaseOff& ph = bs->ph[l];
    ph.gid_begin = bs->G;
    for (int p = 0; p < n_problems; ++p) {
      Problem& P = bs->prob[p];
      if (l >= P.L) continue;
      LevelInfo& L = P.lev[l];
      const bool has_nonleaf = std::any_of(L.leaf.begin(), L.leaf.end(), [](uint8_t v) { return v == 0; });
      for (int variant = 0; variant < (has_nonleaf ? 2 : 1); ++variant) {
        Inst in;
        in.p = p;
        in.l = l;
        in.variant = variant;
        in.h = L.h;
        int rc = build_octree(in, L.c, ctx->max_oct, err);
        if (rc != FLGF_OK) return bail(rc, err);
        in.gid0.resize(in.lv.size());
        in.is_src.resize(in.lv.size());
        in.need_tgt.resize(in.lv.size());
        for (size_t k = 0; k < in.lv.size(); ++k) {
          in.gid0[k] = bs->G;
          bs->G += (int)in.lv[k].size();
          in.is_src[k].assign(in.lv[k].size(), 1);
          in.need_tgt[k].assign(in.lv[k].size(), 0);
        }
        if (variant == 0) {  // targets: the wanted blocks and their octree ancestors
          for (size_t b = 0; b < L.c.size(); ++b) {
            if (!L.want[b]) continue;
            I3 c = L.c[b];
            for (size_t k = 0; k < in.lv.size(); ++k) {
              in.need_tgt[k][in.idx[k][key3(c)]] = 1;
              c = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
            }
          }
        }
        if (variant == 1) {
          for (size_t b = 0; b < L.c.size(); ++b) {
            in.is_src[0][b] = L.leaf[b];
            if (L.ext[b]) {  // target: non-leaf blocks, their buffer, and the ancestors
              I3 c = L.c[b];
              for (size_t k = 0; k < in.lv.size(); ++k) {
                in.need_tgt[k][in.idx[k][key3(c)]] = 1;
                c = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
              }
            }
          }
          L.inst1 = (int)bs->inst.size();
        } else {
          L.inst0 = (int)bs->inst.size();
          L.ugid0 = in.gid0[0];
        }
        bs->inst.push_back(std::move(in));
      }
    }
    ph.nblocks = bs->G - ph.gid_begin;
    bs->max_phase_blocks = std::max(bs->max_phase_blocks, ph.nblocks);
  }
  // pair-list entries hold a phase-local block id in 22 bits
  if (bs->max_phase_blocks >= (1 << 22))
    return bail(FLGF_EINVAL, "more than 2^22 octree blocks in one refinement level");
  // ---- launch lists ----------------------------------------------------------
  Arena& ar = bs->ar;
  for (int l = 0; l < bs->Lmax; ++l) {
    PhaseOff& ph = bs->ph[l];
    std::vector<const Inst*> insts;
    for (const auto& in : bs->inst)
      if (in.l == l) insts.push_back(&in);
    build_fmm(bs, ar, l, insts, ph, true, bs->ncomp);
    // multi-resolution coupling lists
    std::vector<int> sel_src, sel_dst, selw_src, selw_dst, acc_nbr, acc_fine, acc_cpos, accw_nbr, accw_fine,
        accw_cpos, cor_nbr, cor_fine, cor_cpos, crs_c, crs_f;
    std::vector<double> cor_ih2;
    for (int p = 0; p < n_problems; ++p) {
      Problem& P = bs->prob[p];
      if (l >= P.L) continue;
      LevelInfo& L = P.lev[l];
      if (L.inst1 >= 0) {
        const Inst& i1 = bs->inst[L.inst1];
        for (size_t b = 0; b < L.c.size(); ++b) {
          if (!L.leaf[b]) {  // u on non-leaf blocks: the leaf-source field
            sel_src.push_back(i1.gid0[0] + (int)b);
            sel_dst.push_back(L.ugid0 + (int)b);
          }
          if (L.ext[b]) {  // W^l on non-leaf blocks and their buffer
            selw_src.push_back(i1.gid0[0] + (int)b);
            selw_dst.push_back(L.fw0 + (int)b);
          }
        }
      }
      // coarse neighbourhood of a parent as indices into W (level-block numbering)
      auto nbr27 = [&](const LevelInfo& C, const I3& parent, std::vector<int>& outv) {
        for (int e = 0; e < 27; ++e) {
          auto it = C.idx.find(key3(parent[0] + e / 9 - 1, parent[1] + (e / 3) % 3 - 1, parent[2] + e % 3 - 1));
          outv.push_back(it == C.idx.end() ? -1 : C.fw0 + it->second);
        }
      };
      if (l > 0) {
        const LevelInfo& C = P.lev[l - 1];
        for (size_t b = 0; b < L.c.size(); ++b) {
          const I3& c = L.c[b];
          const I3 par = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
          const int cp = ((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1);
          nbr27(C, par, acc_nbr);
          acc_fine.push_back(L.ugid0 + (int)b);
          acc_cpos.push_back(cp);
          if (L.ext[b]) {
            nbr27(C, par, accw_nbr);
            accw_fine.push_back(L.fw0 + (int)b);
            accw_cpos.push_back(cp);
          }
        }
      }
      if (l + 1 < P.L) {
        const LevelInfo& F = P.lev[l + 1];
        for (size_t b = 0; b < F.c.size(); ++b) {
          const I3& c = F.c[b];
          nbr27(L, {c[0] >> 1, c[1] >> 1, c[2] >> 1}, cor_nbr);
          cor_fine.push_back(F.fw0 + (int)b);
          cor_cpos.push_back(((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1));
          cor_ih2.push_back(1.0 / (F.h * F.h));
        }
        for (size_t b = 0; b < L.c.size(); ++b) {
          if (L.leaf[b]) continue;
          crs_c.push_back(L.fw0 + (int)b);
          const I3& c = L.c[b];
          for (int a = 0; a < 8; ++a)
            crs_f.push_back(F.fw0 + F.idx.at(key3(2 * c[0] + (a >> 2), 2 * c[1] + ((a >> 1) & 1), 2 * c[2] + (a & 1))));
        }
      }
    }
    ph.n_sel = (int)sel_src.size();
    ph.sel_src = ar.add(sel_src);
    ph.sel_dst = ar.add(sel_dst);
    ph.n_selw = (int)selw_src.size();
    ph.selw_src = ar.add(selw_src);
    ph.selw_dst = ar.add(selw_dst);
    ph.n_acc = (int)acc_fine.size();
    ph.acc_nbr = ar.add(acc_nbr);
    ph.acc_fine = ar.add(acc_fine);
    ph.acc_cpos = ar.add(acc_cpos);
    ph.n_accw = (int)accw_fine.size();
    ph.accw_nbr = ar.add(accw_nbr);
    ph.accw_fine = ar.add(accw_fine);
    ph.accw_cpos = ar.add(accw_cpos);
    ph.n_cor = (int)cor_fine.size();
    ph.cor_nbr = ar.add(cor_nbr);
    ph.cor_fine = ar.add(cor_fine);
    ph.cor_cpos = ar.add(cor_cpos);
    ph.cor_ih2 = ar.add(cor_ih2);
    ph.n_crs = (int)crs_c.size();
    ph.crs_coarse = ar.add(crs_c);
    ph.crs_fine = ar.add(crs_f);
  }
  // face neighbours for the Laplacian
  for (auto& P : bs->prob)
    for (auto& L : P.lev) {
      std::vector<int> n6;
      for (const auto& c : L.c)
        for (int a = 0; a < 3; ++a)
          for (int sg = 0; sg < 2; ++sg) {
            I3 y = c;
            y[a] += sg == 0 ? 1 : -1;
            auto it = L.idx.find(key3(y));
            n6.push_back(it == L.idx.end() ? -1 : it->second);
          }
      L.nbr6_off = ar.add(n6);
    }
  return FLGF_OK;
}

static int blockset_create(flgf_ctx* ctx, int n_problems, const int* n_levels, const int* nblk,
                           const int32_t* coords, const double* h0, const uint8_t* want, int ncomp,
                           flgf_blockset** out) {
  if (!ctx || !out || n_problems < 1 || !n_levels || !nblk || !coords || !h0)
    return fail(ctx, FLGF_EINVAL, "blockset_create: bad arguments");
  *out = nullptr;
  auto bs = new (std::nothrow) flgf_blockset();
  if (!bs) return fail(ctx, FLGF_ENOMEM, "host allocation");
  bs->ctx = ctx;
  bs->ncomp = ncomp;
  auto bail = [&](int code, const std::string& m) {
    flgf_blockset_destroy(bs);
    return fail(ctx, code, m);
  };
  const int rc = plan_blockset(ctx, bs, n_problems, n_levels, nblk, coords, h0, want);
  if (rc != FLGF_OK) {
    flgf_blockset_destroy(bs);
    return rc;
  }
  bs->compensated = ctx->prec == FLGF_FP32 && bs->Lmax >= 2;
  for (const auto& P : bs->prob)
    for (const auto& L : P.lev)
      bs->masked |= std::any_of(L.want.begin(), L.want.end(), [](uint8_t v) { return v == 0; });
  const int N = ctx->N;
  const size_t N3 = (size_t)N * N * N;
  Arena& ar = bs->ar;
  // ---- device memory ---------------------------------------------------------
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4;
  const size_t NW = (size_t)nfreq(N);
  auto alloc = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes); };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = alloc((void**)&ar.dev, ar.host.size());
  if (e == cudaSuccess) e = cudaMemcpy(ar.dev, ar.host.data(), ar.host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = alloc(&bs->nodes, rs * N3 * bs->G);
  if (e == cudaSuccess) e = alloc(&bs->unodes, rs * N3 * bs->G);
  if (e == cudaSuccess) e = alloc(&bs->fuser, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->fwork, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->wfield, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->spec, 2 * rs * NW * bs->max_phase_blocks);
  if (e == cudaSuccess) e = alloc(&bs->acc, 2 * rs * NW * bs->max_phase_blocks);
  if (e == cudaSuccess) e = alloc(&bs->lap_in, rs * N3 * bs->max_level_blocks);
  if (e == cudaSuccess) e = alloc(&bs->lap_out, rs * N3 * bs->max_level_blocks);
  if (e == cudaSuccess) e = alloc((void**)&bs->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bs->fuser, 0, rs * N3 * bs->B);
  if (e == cudaSuccess) e = cudaMemset(bs->unodes, 0, rs * N3 * bs->G);
  if (e == cudaSuccess) e = cudaMemset(bs->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs->cstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->ev_fuser_free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->ev_loaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bs->ev_dev_load, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? FLGF_ENOMEM : FLGF_ECUDA;
    return bail(code, std::string("blockset allocation: ") + cudaGetErrorString(e));
  }
  *out = bs;
  return FLGF_OK;
}

extern "C" int flgf_blockset_create(flgf_ctx* ctx, int n_problems, const int* n_levels, const int* nblk,
                                    const int32_t* coords, const double* h0, flgf_blockset** out) {
  return blockset_create(ctx, n_problems, n_levels, nblk, coords, h0, nullptr, 1, out);
}

extern "C" int flgf_blockset_create_masked(flgf_ctx* ctx, int n_problems, const int* n_levels, const int* nblk,
                                           const int32_t* coords, const double* h0, const uint8_t* want,
                                           flgf_blockset** out) {
  return blockset_create(ctx, n_problems, n_levels, nblk, coords, h0, want, 1, out);
}

extern "C" int flgf_blockset_create_vector(flgf_ctx* ctx, int n_components, int n_levels, const int* nblk,
                                           const int32_t* coords, double h0, flgf_blockset** out) {
  if (!ctx || !out || n_components < 1 || n_components > 64 || n_levels < 1 || !nblk || !coords)
    return fail(ctx, FLGF_EINVAL, "blockset_create_vector: bad arguments");
  int64_t nb = 0;
  for (int l = 0; l < n_levels; ++l) {
    if (nblk[l] < 0) return fail(ctx, FLGF_EINVAL, "blockset_create_vector: negative block count");
    nb += nblk[l];
  }
  // the components as problems on copies of one mesh
  std::vector<int> nlev(n_components, n_levels), nb_all;
  std::vector<int32_t> c_all;
  std::vector<double> h_all(n_components, h0);
  try {
    nb_all.reserve((size_t)n_components * n_levels);
    c_all.reserve((size_t)n_components * 3 * nb);
    for (int c = 0; c < n_components; ++c) {
      nb_all.insert(nb_all.end(), nblk, nblk + n_levels);
      c_all.insert(c_all.end(), coords, coords + 3 * nb);
    }
  } catch (const std::bad_alloc&) {
    return fail(ctx, FLGF_ENOMEM, "host allocation");
  }
  return blockset_create(ctx, n_components, nlev.data(), nb_all.data(), c_all.data(), h_all.data(), nullptr,
                         n_components, out);
}

// Adjoint plan, built on first use: the transposed leaf-only instances, their
// FMM lists and the transposed coupling lists (in their own arena), and the
// adjoint buffers.  Forward-only users pay neither its host time nor its
// device memory.
static int build_adjoint(flgf_blockset* bs) {
  flgf_ctx* ctx = bs->ctx;
  // the adjoint reuses the forward lists, which a target mask has pruned
  if (bs->masked) return fail(ctx, FLGF_ESTATE, "the adjoint needs a block set without a target mask");
  const size_t N3 = (size_t)ctx->N * ctx->N * ctx->N;
  // start from nothing, so a call after a failed one (out of memory) rebuilds cleanly
  for (void** p : {&bs->gseed, &bs->gW, &bs->gf, &bs->gtmp, &bs->aunodes}) {
    cudaFree(*p);
    *p = nullptr;
  }
  cudaFree(bs->aar.dev);
  bs->aar = Arena();
  bs->aph.assign(bs->Lmax, PhaseOff());
  bs->adj.assign(bs->Lmax, AdjOff());
  bs->adj_inst.clear();
  Arena& aar = bs->aar;
  bs->adj_inst.reserve(bs->inst.size());
  for (const auto& in : bs->inst) {
    if (in.variant != 1) continue;
    Inst t = in;  // same octree and global ids as the forward leaf-only instance
    const LevelInfo& L = bs->prob[in.p].lev[in.l];
    for (size_t k = 0; k < t.lv.size(); ++k) t.need_tgt[k].assign(t.lv[k].size(), 0);
    for (size_t b = 0; b < L.c.size(); ++b) {
      t.is_src[0][b] = L.ext[b];
      if (L.leaf[b]) {
        I3 c = L.c[b];
        for (size_t k = 0; k < t.lv.size(); ++k) {
          t.need_tgt[k][t.idx[k][key3(c)]] = 1;
          c = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
        }
      }
    }
    t.variant = 2;
    bs->adj_inst.push_back(std::move(t));
  }
  for (int l = 0; l < bs->Lmax; ++l) {
    std::vector<const Inst*> insts;
    for (const auto& in : bs->inst)
      if (in.l == l && in.variant == 0) insts.push_back(&in);
    for (const auto& in : bs->adj_inst)
      if (in.l == l) insts.push_back(&in);
    bs->aph[l].gid_begin = bs->ph[l].gid_begin;
    bs->aph[l].nblocks = bs->ph[l].nblocks;
    build_fmm(bs, aar, l, insts, bs->aph[l], false, 1);
    AdjOff& ao = bs->adj[l];
    std::vector<int> pd, p1, p2, gd, g1, g2, td, t1, t2, c0n, c0f, c0c, c1n, c1f, c1c;
    std::vector<double> c1h;
    for (int p = 0; p < (int)bs->prob.size(); ++p) {
      Problem& P = bs->prob[p];
      if (l >= P.L) continue;
      LevelInfo& L = P.lev[l];
      const Inst& i0 = bs->inst[L.inst0];
      const bool has1 = L.inst1 >= 0;
      const int g1base = has1 ? bs->inst[L.inst1].gid0[0] : -1;
      for (size_t b = 0; b < L.c.size(); ++b) {
        const int fb = L.fw0 + (int)b;
        pd.push_back(i0.gid0[0] + (int)b);  // A^T applied to the leaf part of the adjoint of u
        p1.push_back(L.leaf[b] ? fb : -1);
        p2.push_back(-1);
        if (has1) {                          // A^T (P_leaf) applied to the adjoint of the leaf-source field
          pd.push_back(g1base + (int)b);
          p1.push_back(L.leaf[b] ? -1 : fb);
          p2.push_back(L.ext[b] ? fb : -1);
        }
        gd.push_back(fb);
        g1.push_back(i0.gid0[0] + (int)b);
        g2.push_back(has1 && L.leaf[b] ? g1base + (int)b : -1);
        if (l > 0) {
          td.push_back(fb);
          t1.push_back(fb);
          t2.push_back(L.ext[b] ? fb : -1);
        }
      }
      auto nbr27 = [&](const LevelInfo& C, const I3& parent, std::vector<int>& outv) {
        for (int e = 0; e < 27; ++e) {
          auto it = C.idx.find(key3(parent[0] + e / 9 - 1, parent[1] + (e / 3) % 3 - 1, parent[2] + e % 3 - 1));
          outv.push_back(it == C.idx.end() ? -1 : C.fw0 + it->second);
        }
      };
      if (l > 0) {
        const LevelInfo& C = P.lev[l - 1];
        for (size_t b = 0; b < L.c.size(); ++b) {
          const I3& c = L.c[b];
          nbr27(C, {c[0] >> 1, c[1] >> 1, c[2] >> 1}, c0n);
          c0f.push_back(L.fw0 + (int)b);
          c0c.push_back(((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1));
        }
      }
      if (l + 1 < P.L) {
        const LevelInfo& Fl = P.lev[l + 1];
        for (size_t b = 0; b < Fl.c.size(); ++b) {
          const I3& c = Fl.c[b];
          nbr27(L, {c[0] >> 1, c[1] >> 1, c[2] >> 1}, c1n);
          c1f.push_back(Fl.fw0 + (int)b);
          c1c.push_back(((c[0] & 1) << 2) | ((c[1] & 1) << 1) | (c[2] & 1));
          c1h.push_back(1.0 / (Fl.h * Fl.h));
        }
      }
    }
    ao.n_prep = (int)pd.size(); ao.prep_dst = aar.add(pd); ao.prep_s1 = aar.add(p1); ao.prep_s2 = aar.add(p2);
    ao.n_gacc = (int)gd.size(); ao.gacc_dst = aar.add(gd); ao.gacc_s1 = aar.add(g1); ao.gacc_s2 = aar.add(g2);
    ao.n_gtmp = (int)td.size(); ao.gtmp_dst = aar.add(td); ao.gtmp_s1 = aar.add(t1); ao.gtmp_s2 = aar.add(t2);
    ao.n_cf0 = (int)c0f.size(); ao.cf0_nbr = aar.add(c0n); ao.cf0_fine = aar.add(c0f); ao.cf0_cpos = aar.add(c0c);
    ao.n_cf1 = (int)c1f.size(); ao.cf1_nbr = aar.add(c1n); ao.cf1_fine = aar.add(c1f); ao.cf1_cpos = aar.add(c1c);
    ao.cf1_ih2 = aar.add(c1h);
  }
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4;
  auto alloc = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes); };
  cudaError_t e = alloc((void**)&aar.dev, aar.host.size());
  if (e == cudaSuccess) e = cudaMemcpy(aar.dev, aar.host.data(), aar.host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = alloc(&bs->gseed, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->gW, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->gf, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->gtmp, rs * N3 * bs->B);
  if (e == cudaSuccess) e = alloc(&bs->aunodes, rs * N3 * bs->G);
  if (e == cudaSuccess) e = cudaMemset(bs->gseed, 0, rs * N3 * bs->B);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? FLGF_ENOMEM : FLGF_ECUDA;
    return fail(ctx, code, std::string("adjoint allocation: ") + cudaGetErrorString(e));
  }
  bs->adj_ready = true;
  return FLGF_OK;
}

extern "C" int64_t flgf_blockset_dof(const flgf_blockset* bs) { return bs ? bs->dof : -1; }

extern "C" int64_t flgf_launch_count(const flgf_blockset* bs) { return bs ? bs->launches : -1; }

extern "C" int flgf_work_counts(const flgf_blockset* bs, int64_t* pairs, int64_t* fwd, int64_t* inv, int64_t* koff) {
  if (!bs) return FLGF_EINVAL;
  if (pairs) *pairs = bs->pairs;
  if (fwd) *fwd = bs->n_fwd;
  if (inv) *inv = bs->n_inv;
  if (koff) *koff = bs->n_koff;
  return FLGF_OK;
}

namespace {

int check_pl(flgf_blockset* bs, int problem, int level) {
  if (problem < 0 || problem >= (int)bs->prob.size()) return FLGF_EINVAL;
  if (level < 0 || level >= bs->prob[problem].L) return FLGF_EINVAL;
  return FLGF_OK;
}

cudaMemcpyKind kind(int where, bool to_dev) {
  if (where == FLGF_DEVICE) return cudaMemcpyDeviceToDevice;
  return to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

}  // namespace

extern "C" int flgf_load_source(flgf_blockset* bs, int problem, int level, const void* f, int where) {
  if (!bs || !f || (where != FLGF_HOST && where != FLGF_DEVICE)) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (check_pl(bs, problem, level) != FLGF_OK) return fail(ctx, FLGF_EINVAL, "load_source: bad problem/level");
  const LevelInfo& L = bs->prob[problem].lev[level];
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4, N3 = (size_t)ctx->N * ctx->N * ctx->N;
  char* dst = (char*)bs->fuser + rs * N3 * L.fw0;
  const size_t bytes = rs * N3 * L.c.size();
  if (where == FLGF_HOST) {
    // on the copy stream, after the last solve has taken its copy of the source
    // buffer and after earlier device loads; returns once the copy is done
    CK(cudaStreamWaitEvent(bs->cstream, bs->ev_fuser_free, 0));
    CK(cudaStreamWaitEvent(bs->cstream, bs->ev_dev_load, 0));
    CK(cudaMemcpyAsync(dst, f, bytes, cudaMemcpyHostToDevice, bs->cstream));
    CK(cudaEventRecord(bs->ev_loaded, bs->cstream));
    CK(cudaEventSynchronize(bs->ev_loaded));
    bs->load_pending = true;
  } else {
    if (bs->load_pending) CK(cudaStreamWaitEvent(ctx->stream, bs->ev_loaded, 0));
    CK(cudaMemcpyAsync(dst, f, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaEventRecord(bs->ev_dev_load, ctx->stream));
  }
  return FLGF_OK;
}

// ----------------------------------------------------------------------------
// Solve
// ----------------------------------------------------------------------------
namespace {

struct StageScope {
  flgf_blockset* bs;
  int stage;
  cudaEvent_t end = nullptr;
  StageScope(flgf_blockset* b, int s) : bs(b), stage(s) {
    if (!bs->timing) return;
    if (bs->ev_used == bs->ev.size()) {
      cudaEvent_t a, c;
      cudaEventCreate(&a);
      cudaEventCreate(&c);
      bs->ev.push_back({s, {a, c}});
    }
    auto& slot = bs->ev[bs->ev_used++];
    slot.first = s;
    record(slot.second.first);
    end = slot.second.second;
  }
  // Inside stream capture a plain record only orders work; an external
  // record node is needed for the event to be timed when the graph runs.
  void record(cudaEvent_t e) const {
    if (bs->capturing)
      cudaEventRecordWithFlags(e, bs->ctx->stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, bs->ctx->stream);
  }
  ~StageScope() {
    if (end) record(end);
  }
};

// FMM of one phase: upward pass over `nodes`, forward FFTs, spectrum MAC,
// inverse FFTs and downward pass into `unodes`.
template <typename R>
cudaError_t enqueue_fmm(flgf_blockset* bs, const Arena& ar, const PhaseOff& ph, R* unodes) {
  flgf_ctx* c = bs->ctx;
  const int N = c->N;
  cudaStream_t s = c->stream;
  R* nodes = (R*)bs->nodes;
  cudaError_t e;
#define KRUN(n, x)                              \
  do {                                          \
    if ((n) > 0) bs->launches++;                \
    if ((e = (x)) != cudaSuccess) return e;     \
  } while (0)
  const int maxtop = (int)ph.n_ant.size() - 1;
  {
    StageScope sc(bs, 1);
    for (int k = 1; k <= maxtop; ++k)
      KRUN(ph.n_ant[k], launch_anterp<R>(N, c->nI, c->d_J1, ar.at<int>(ph.ant_par[k]), ar.at<int>(ph.ant_ch[k]),
                                         ph.n_ant[k], nodes, s));
  }
  // The fields of the octree levels above the finest are extrapolated to the
  // outer faces of the child blocks by the downward pass, whose Lagrange rows
  // there amplify white rounding noise ~38x at a block corner (n_I = 6).  With
  // FLGF_OPT_COMPENSATED an FP32 block set therefore transforms those levels
  // back (inverse FFT) and interpolates in float-float arithmetic; the finest
  // level's inverse FFTs, which nothing amplifies, stay plain FP32.
  const bool comp = bs->compensated;
  {
    StageScope sc(bs, 2);
    KRUN(ph.n_fwd, launch_fft_forward<R>(N, nodes, ar.at<int>(ph.fwd_gid), ar.at<int>(ph.fwd_sid), ph.n_fwd, bs->spec,
                                         ph.nblocks, s));
  }
  {
    StageScope sc(bs, 3);
    KRUN(ph.n_work, launch_hadamard<R>(N, ar.at<HadGroup>(ph.hgroups), ar.at<HadWork>(ph.work), ph.n_work,
                                       ph.max_units, ar.at<int>(ph.src_ids), ar.at<int>(ph.tgt_ids),
                                       ar.at<uint16_t>(ph.par_tab), bs->spec, bs->acc, ph.nblocks, c->d_kspec,
                                       c->kstride, s));
    KRUN(ph.n_fl, launch_hadamard_fl(N, ar.at<FlGroup>(ph.fl_groups), ph.n_fl, ph.fl_max_cells, ph.fl_max_parents,
                                     ar.at<uint16_t>(ph.fl_rows), ar.at<uint32_t>(ph.fl_dlms), ar.at<int>(ph.fl_tgt),
                                     ar.at<int>(ph.fl_cells), bs->spec, bs->acc, ph.nblocks, c->d_kspec, c->kstride,
                                     ph.fl_ncomp, ph.fl_cstride, ph.fl_split, s));
    KRUN(ph.n_fll, launch_hadamard_fll(N, ar.at<FllGroup>(ph.fll_groups), ph.n_fll, ar.at<int>(ph.fll_tgt),
                                       ar.at<int>(ph.fll_beg), ar.at<int>(ph.fll_len), ar.at<uint32_t>(ph.fll_ent),
                                       bs->spec, bs->acc, ph.nblocks, c->d_kspec, c->kstride, s));
    KRUN(ph.n_groups, launch_hadamard_list<R>(N, ar.at<ListGroup>(ph.groups), ph.n_groups, ph.max_group_src,
                                              ar.at<int>(ph.l_tgt), ar.at<int>(ph.l_len), ar.at<int>(ph.l_ent),
                                              ar.at<int>(ph.l_src), bs->spec, bs->acc, ph.nblocks, c->d_kspec,
                                              c->kstride, s));
  }
  {
    StageScope sc(bs, 4);
    KRUN(ph.n_inv0, launch_fft_inverse<R>(N, bs->acc, ph.nblocks, ar.at<int>(ph.inv_sid), ar.at<int>(ph.inv_gid),
                                          ar.at<double>(ph.inv_scale), ph.n_inv0, unodes, s, false));
    const int nc = ph.n_inv - ph.n_inv0;
    KRUN(nc, launch_fft_inverse<R>(N, bs->acc, ph.nblocks, ar.at<int>(ph.inv_sid) + ph.n_inv0,
                                   ar.at<int>(ph.inv_gid) + ph.n_inv0, ar.at<double>(ph.inv_scale) + ph.n_inv0, nc,
                                   unodes, s, comp));
  }
  {
    StageScope sc(bs, 5);
    for (int k = maxtop - 1; k >= 0; --k)
      KRUN(ph.n_itp[k], launch_interp_add<R>(N, c->nI, c->d_J1, ar.at<int>(ph.itp_ch[k]), ar.at<int>(ph.itp_par[k]),
                                             ar.at<int>(ph.itp_cpos[k]), ph.n_itp[k], unodes, s, comp));
  }
#undef KRUN
  return cudaSuccess;
}

// Adjoint of the solve: the transposes of Sec. 3's steps in reverse order
// (correction, FMMs -- symmetric, with source and target masks swapped for
// the leaf-only one -- selection, accumulation, then the coarsening).
template <typename R>
cudaError_t enqueue_adjoint(flgf_blockset* bs) {
  flgf_ctx* c = bs->ctx;
  const int N = c->N;
  cudaStream_t s = c->stream;
  const Arena& ar = bs->ar;   // forward lists (coarsening)
  const Arena& aa = bs->aar;  // adjoint lists
  const size_t N3 = (size_t)N * N * N;
  R* nodes = (R*)bs->nodes;
  R* unodes = (R*)bs->aunodes;
  R* gseed = (R*)bs->gseed;
  R* gW = (R*)bs->gW;
  R* gf = (R*)bs->gf;
  R* gtmp = (R*)bs->gtmp;
  cudaError_t e;
#define RUN(x) \
  if ((e = (x)) != cudaSuccess) return e;
#define KRUN(n, x)                              \
  do {                                          \
    if ((n) > 0) bs->launches++;                \
    if ((e = (x)) != cudaSuccess) return e;     \
  } while (0)
  bs->launches = 0;
  RUN(cudaMemsetAsync(bs->d_err, 0, sizeof(int), s));
  RUN(cudaMemsetAsync(gW, 0, sizeof(R) * N3 * bs->B, s));
  RUN(cudaMemsetAsync(gf, 0, sizeof(R) * N3 * bs->B, s));
  for (int l = bs->Lmax - 1; l >= 0; --l) {
    const AdjOff& ao = bs->adj[l];
    {
      StageScope sc(bs, 6);
      if (bs->correction)
        KRUN(ao.n_cf1, launch_cf_interp_adjoint<R>(N, gW, aa.at<int>(ao.cf1_nbr), gf, aa.at<int>(ao.cf1_fine),
                                                   aa.at<int>(ao.cf1_cpos), ao.n_cf1, 1, aa.at<double>(ao.cf1_ih2),
                                                   bs->d_err, s));
      KRUN(ao.n_prep, launch_combine_blocks<R>(N, nodes, aa.at<int>(ao.prep_dst), gseed, aa.at<int>(ao.prep_s1), gW,
                                               aa.at<int>(ao.prep_s2), 0, ao.n_prep, s));
    }
    if ((e = enqueue_fmm<R>(bs, aa, bs->aph[l], unodes)) != cudaSuccess) return e;
    {
      StageScope sc(bs, 6);
      KRUN(ao.n_gacc, launch_combine_blocks<R>(N, gf, aa.at<int>(ao.gacc_dst), unodes, aa.at<int>(ao.gacc_s1), unodes,
                                               aa.at<int>(ao.gacc_s2), 1, ao.n_gacc, s));
      KRUN(ao.n_gtmp, launch_combine_blocks<R>(N, gtmp, aa.at<int>(ao.gtmp_dst), gseed, aa.at<int>(ao.gtmp_s1), gW,
                                               aa.at<int>(ao.gtmp_s2), 0, ao.n_gtmp, s));
      KRUN(ao.n_cf0, launch_cf_interp_adjoint<R>(N, gW, aa.at<int>(ao.cf0_nbr), gtmp, aa.at<int>(ao.cf0_fine),
                                                 aa.at<int>(ao.cf0_cpos), ao.n_cf0, 0, nullptr, bs->d_err, s));
    }
  }
  {
    StageScope sc(bs, 0);
    for (int l = 0; l + 1 < bs->Lmax; ++l) {
      const PhaseOff& ph = bs->ph[l];
      KRUN(ph.n_crs, launch_coarsen_adjoint<R>(N, gf, ar.at<int>(ph.crs_fine), ar.at<int>(ph.crs_coarse), ph.n_crs, s));
    }
  }
#undef KRUN
#undef RUN
  return cudaSuccess;
}

template <typename R>
cudaError_t enqueue_solve(flgf_blockset* bs) {
  flgf_ctx* c = bs->ctx;
  const int N = c->N;
  cudaStream_t s = c->stream;
  const Arena& ar = bs->ar;
  R* nodes = (R*)bs->nodes;
  R* unodes = (R*)bs->unodes;
  R* fwork = (R*)bs->fwork;
  const size_t N3 = (size_t)N * N * N;
  cudaError_t e;
#define RUN(x)                              \
  if ((e = (x)) != cudaSuccess) return e;
#define KRUN(n, x)                              \
  do {                                          \
    if ((n) > 0) bs->launches++;                \
    if ((e = (x)) != cudaSuccess) return e;     \
  } while (0)
  bs->launches = 0;
  RUN(cudaMemsetAsync(bs->d_err, 0, sizeof(int), s));
  RUN(cudaMemcpyAsync(fwork, bs->fuser, sizeof(R) * N3 * bs->B, cudaMemcpyDeviceToDevice, s));
  RUN(cudaEventRecordWithFlags(bs->ev_fuser_free, s, bs->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  {
    StageScope sc(bs, 0);
    for (int l = bs->Lmax - 2; l >= 0; --l) {
      const PhaseOff& ph = bs->ph[l];
      KRUN(ph.n_crs, launch_coarsen<R>(N, fwork, ar.at<int>(ph.crs_fine), fwork, ar.at<int>(ph.crs_coarse), ph.n_crs, s));
    }
  }
  for (int l = 0; l < bs->Lmax; ++l) {
    const PhaseOff& ph = bs->ph[l];
    const int maxtop = (int)ph.n_ant.size() - 1;
    {
      StageScope sc(bs, 1);
      KRUN(ph.n_prep, launch_copy_blocks<R>(N, fwork, ar.at<int>(ph.prep_src), nodes, ar.at<int>(ph.prep_dst),
                                            ar.at<uint8_t>(ph.prep_zero), ph.n_prep, s));
    }
    if ((e = enqueue_fmm<R>(bs, bs->ar, ph, unodes)) != cudaSuccess) return e;
    {
      StageScope sc(bs, 6);
      R* wf = (R*)bs->wfield;
      KRUN(ph.n_sel, launch_copy_blocks<R>(N, unodes, ar.at<int>(ph.sel_src), unodes, ar.at<int>(ph.sel_dst), nullptr,
                                           ph.n_sel, s));
      KRUN(ph.n_selw, launch_copy_blocks<R>(N, unodes, ar.at<int>(ph.selw_src), wf, ar.at<int>(ph.selw_dst), nullptr,
                                            ph.n_selw, s));
      // accumulation from the coarser level's leaf-source field W^{l-1}
      KRUN(ph.n_acc, launch_cf_interp<R>(N, wf, ar.at<int>(ph.acc_nbr), ar.at<int>(ph.acc_fine), ar.at<int>(ph.acc_cpos),
                                         ph.n_acc, unodes, 0, nullptr, bs->d_err, s));
      KRUN(ph.n_accw, launch_cf_interp<R>(N, wf, ar.at<int>(ph.accw_nbr), ar.at<int>(ph.accw_fine),
                                          ar.at<int>(ph.accw_cpos), ph.n_accw, wf, 0, nullptr, bs->d_err, s));
      if (bs->correction)
        KRUN(ph.n_cor, launch_cf_interp<R>(N, wf, ar.at<int>(ph.cor_nbr), ar.at<int>(ph.cor_fine), ar.at<int>(ph.cor_cpos),
                                           ph.n_cor, fwork, 1, ar.at<double>(ph.cor_ih2), bs->d_err, s));
    }
  }
#undef KRUN
#undef RUN
  return cudaSuccess;
}

void collect_times(flgf_blockset* bs) {
  if (!bs->ev_pending) return;
  cudaStreamSynchronize(bs->ctx->stream);
  for (size_t i = 0; i < bs->ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, bs->ev[i].second.first, bs->ev[i].second.second) == cudaSuccess)
      bs->stage_ms[bs->ev[i].first] += ms;
    else
      (void)cudaGetLastError();  // a missing timing must not poison later calls
  }
  bs->timed_solves++;
  bs->ev_pending = false;
}

}  // namespace

extern "C" int flgf_ctx_set_option(flgf_ctx* ctx, int key, int value) {
  if (!ctx) return FLGF_EINVAL;
  switch (key) {
    case FLGF_CTX_LIST_PCT:
      if (value < 0 || value > 100) return fail(ctx, FLGF_EINVAL, "list percentage must be 0..100");
      ctx->list_pct = value;
      return FLGF_OK;
    case FLGF_CTX_MAC:
      if (value < 0 || value > 2) return fail(ctx, FLGF_EINVAL, "FLGF_CTX_MAC takes 0, 1 or 2");
      ctx->mac = value;
      return FLGF_OK;
    case FLGF_CTX_ORDER:
      if (value != 0 && value != 1) return fail(ctx, FLGF_EINVAL, "FLGF_CTX_ORDER takes 0 or 1");
      ctx->order_by_list = value == 1;
      return FLGF_OK;
    case FLGF_CTX_FAIL_ALLOC:
      if (value < 0) return fail(ctx, FLGF_EINVAL, "allocation failure index must be >= 0");
      ctx->fail_alloc_at = value;
      ctx->alloc_count = 0;
      return FLGF_OK;
    case FLGF_CTX_TILE: {
      const int t[3] = {value & 255, (value >> 8) & 255, (value >> 16) & 255};
      for (int a = 0; a < 3; ++a)
        if (t[a] < 1 || t[a] > 8) return fail(ctx, FLGF_EINVAL, "tile extents must be 1..8 parents");
      if (value >> 24 || t[0] * t[1] * t[2] > 128 || (t[0] + 2) * (t[1] + 2) * (t[2] + 2) > 397)
        return fail(ctx, FLGF_EINVAL, "tile too large for the spectrum MAC");
      for (int a = 0; a < 3; ++a) ctx->tile[a] = t[a];
      return FLGF_OK;
    }
    default:
      return fail(ctx, FLGF_EINVAL, "unknown context option");
  }
}

extern "C" int flgf_set_option(flgf_blockset* bs, int key, int value) {
  if (!bs) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  switch (key) {
    case FLGF_OPT_CORRECTION:
      bs->correction = value != 0;
      break;
    case FLGF_OPT_GRAPH:
      if (value && ctx->stream == nullptr)
        return fail(ctx, FLGF_EINVAL, "graph capture needs a non-default stream");
      bs->use_graph = value != 0;
      break;
    case FLGF_OPT_TIMING:
      bs->timing = value != 0;
      break;
    case FLGF_OPT_FAULT_HALO: {
      // failure injection: mark one coarse neighbour of the first coarse-fine
      // accumulation list absent, in the host copy and on the device, as if
      // the mesh lacked that halo block (the kernel then reads zero there and
      // raises the device error flag)
      if (value != 1) return fail(ctx, FLGF_EINVAL, "FLGF_OPT_FAULT_HALO takes 1");
      for (const PhaseOff& ph : bs->ph) {
        if (ph.n_acc == 0) continue;
        int* h = reinterpret_cast<int*>(bs->ar.host.data() + ph.acc_nbr);
        for (int i = 13; i < 27 * ph.n_acc; i += 27) {  // the parent itself: read for every child position
          if (h[i] < 0) continue;
          h[i] = -1;
          CK(cudaMemcpy(bs->ar.dev + ph.acc_nbr + sizeof(int) * i, &h[i], sizeof(int), cudaMemcpyHostToDevice));
          if (bs->gexec) {
            cudaGraphExecDestroy(bs->gexec);
            bs->gexec = nullptr;
          }
          return FLGF_OK;
        }
      }
      return fail(ctx, FLGF_EINVAL, "FLGF_OPT_FAULT_HALO: the block set has no coarse-fine interpolation");
    }
    case FLGF_OPT_COMPENSATED:
      if (value != 0 && value != 1) return fail(ctx, FLGF_EINVAL, "FLGF_OPT_COMPENSATED takes 0 or 1");
      bs->compensated = value == 1 && ctx->prec == FLGF_FP32;
      break;
    default:
      return fail(ctx, FLGF_EINVAL, "unknown option");
  }
  // any change invalidates a captured graph
  if (bs->gexec) {
    cudaGraphExecDestroy(bs->gexec);
    bs->gexec = nullptr;
  }
  return FLGF_OK;
}

extern "C" int flgf_solve(flgf_blockset* bs) {
  if (!bs) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  collect_times(bs);
  cudaError_t e;
  if (bs->load_pending) {  // a host load on the copy stream feeds this solve
    CK(cudaStreamWaitEvent(ctx->stream, bs->ev_loaded, 0));
    bs->load_pending = false;
  }
  if (bs->use_graph) {
    if (!bs->gexec) {
      bs->ev_used = 0;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      bs->capturing = true;
      e = ctx->prec == FLGF_FP64 ? enqueue_solve<double>(bs) : enqueue_solve<float>(bs);
      bs->capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, FLGF_ECUDA, std::string("solve capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&bs->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(bs->gexec, ctx->stream));
  } else {
    bs->ev_used = 0;
    e = ctx->prec == FLGF_FP64 ? enqueue_solve<double>(bs) : enqueue_solve<float>(bs);
    if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
  }
  bs->ev_pending = bs->timing && bs->ev_used > 0;
  bs->solved = true;
  return FLGF_OK;
}

extern "C" int flgf_stage_times(flgf_blockset* bs, double* ms, int n_stages, int* n_solves, int reset) {
  if (!bs || n_stages < 0 || n_stages > 7 || (n_stages > 0 && !ms)) return FLGF_EINVAL;
  collect_times(bs);
  for (int i = 0; i < n_stages; ++i) ms[i] = bs->stage_ms[i];
  if (n_solves) *n_solves = bs->timed_solves;
  if (reset) {
    for (double& v : bs->stage_ms) v = 0.0;
    bs->timed_solves = 0;
  }
  return FLGF_OK;
}

namespace {
// Waits for the context stream and reports the device error flag that the
// kernels of the last solve (forward or adjoint) raise on a missing halo block.
int check_device_flag(flgf_blockset* bs, const char* what) {
  flgf_ctx* ctx = bs->ctx;
  CK(cudaStreamSynchronize(ctx->stream));
  int herr = 0;
  CK(cudaMemcpy(&herr, bs->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return fail(ctx, FLGF_EDEVICE, std::string(what) + ": a coarse-fine interpolation met a missing halo block");
  return FLGF_OK;
}
}  // namespace

extern "C" int flgf_load_adjoint(flgf_blockset* bs, int problem, int level, const void* g, int where) {
  if (!bs || !g || (where != FLGF_HOST && where != FLGF_DEVICE)) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (check_pl(bs, problem, level) != FLGF_OK) return fail(ctx, FLGF_EINVAL, "load_adjoint: bad problem/level");
  if (!bs->adj_ready) {
    const int rc = build_adjoint(bs);
    if (rc != FLGF_OK) return rc;
  }
  const LevelInfo& L = bs->prob[problem].lev[level];
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4, N3 = (size_t)ctx->N * ctx->N * ctx->N;
  CK(cudaMemcpyAsync((char*)bs->gseed + rs * N3 * L.fw0, g, rs * N3 * L.c.size(), kind(where, true), ctx->stream));
  if (where == FLGF_HOST) CK(cudaStreamSynchronize(ctx->stream));
  return FLGF_OK;
}

extern "C" int flgf_solve_adjoint(flgf_blockset* bs) {
  if (!bs) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (!bs->adj_ready) {
    const int rc = build_adjoint(bs);
    if (rc != FLGF_OK) return rc;
  }
  collect_times(bs);
  bs->ev_used = 0;
  cudaError_t e = ctx->prec == FLGF_FP64 ? enqueue_adjoint<double>(bs) : enqueue_adjoint<float>(bs);
  if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("solve_adjoint: ") + cudaGetErrorString(e));
  bs->ev_pending = bs->timing && bs->ev_used > 0;
  bs->adj_solved = true;
  return FLGF_OK;
}

extern "C" int flgf_get_gradient(flgf_blockset* bs, int problem, int level, void* out, int where) {
  if (!bs || !out || (where != FLGF_HOST && where != FLGF_DEVICE)) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (check_pl(bs, problem, level) != FLGF_OK) return fail(ctx, FLGF_EINVAL, "get_gradient: bad problem/level");
  if (!bs->adj_solved) return fail(ctx, FLGF_ESTATE, "get_gradient before solve_adjoint");
  const LevelInfo& L = bs->prob[problem].lev[level];
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4, N3 = (size_t)ctx->N * ctx->N * ctx->N;
  CK(cudaMemcpyAsync(out, (char*)bs->gf + rs * N3 * L.fw0, rs * N3 * L.c.size(), kind(where, false), ctx->stream));
  return check_device_flag(bs, "get_gradient");
}

extern "C" int flgf_get_potential(flgf_blockset* bs, int problem, int level, void* u, int where) {
  if (!bs || !u || (where != FLGF_HOST && where != FLGF_DEVICE)) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (check_pl(bs, problem, level) != FLGF_OK) return fail(ctx, FLGF_EINVAL, "get_potential: bad problem/level");
  if (!bs->solved) return fail(ctx, FLGF_ESTATE, "get_potential before solve");
  const LevelInfo& L = bs->prob[problem].lev[level];
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4, N3 = (size_t)ctx->N * ctx->N * ctx->N;
  CK(cudaMemcpyAsync(u, (char*)bs->unodes + rs * N3 * L.ugid0, rs * N3 * L.c.size(), kind(where, false), ctx->stream));
  return check_device_flag(bs, "get_potential");
}

extern "C" int flgf_laplacian(flgf_blockset* bs, int problem, int level, const void* u, void* out, int where) {
  if (!bs || !u || !out || (where != FLGF_HOST && where != FLGF_DEVICE)) return FLGF_EINVAL;
  flgf_ctx* ctx = bs->ctx;
  if (check_pl(bs, problem, level) != FLGF_OK) return fail(ctx, FLGF_EINVAL, "laplacian: bad problem/level");
  const LevelInfo& L = bs->prob[problem].lev[level];
  const int N = ctx->N;
  const size_t rs = ctx->prec == FLGF_FP64 ? 8 : 4, N3 = (size_t)N * N * N, bytes = rs * N3 * L.c.size();
  const void* din = u;
  void* dout = out;
  if (where == FLGF_HOST) {
    CK(cudaMemcpyAsync(bs->lap_in, u, bytes, cudaMemcpyHostToDevice, ctx->stream));
    din = bs->lap_in;
    dout = bs->lap_out;
  }
  const double ih2 = 1.0 / (L.h * L.h);
  cudaError_t e = ctx->prec == FLGF_FP64
                      ? launch_laplacian<double>(N, (const double*)din, bs->ar.at<int>(L.nbr6_off), (int)L.c.size(), ih2,
                                                 (double*)dout, ctx->stream)
                      : launch_laplacian<float>(N, (const float*)din, bs->ar.at<int>(L.nbr6_off), (int)L.c.size(), ih2,
                                                (float*)dout, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("laplacian: ") + cudaGetErrorString(e));
  if (where == FLGF_HOST) {
    CK(cudaMemcpyAsync(out, bs->lap_out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return FLGF_OK;
}

extern "C" int flgf_refine_level(flgf_ctx* ctx, const void* f, int nblk, const int32_t* coords, double rel,
                                 uint8_t* flags, int32_t* children, int32_t* buffer, int* counts) {
  if (!ctx || !f || !coords || !flags || !children || !buffer || !counts || nblk < 1 || !(rel >= 0.0) ||
      rel > 1e300)
    return fail(ctx, FLGF_EINVAL, "refine_level: bad arguments");
  counts[0] = counts[1] = 0;
  const cudaError_t e = launch_refine_level(ctx->N, ctx->prec == FLGF_FP64, f, nblk, coords, rel, flags, children,
                                            buffer, counts, ctx->stream);
  if (e == cudaErrorInvalidValue)
    return fail(ctx, FLGF_EINVAL, "refine_level: a coordinate outside (-2^19, 2^19) or more than 645277 blocks");
  if (e == cudaErrorMemoryAllocation) return fail(ctx, FLGF_ENOMEM, "refine_level: scratch allocation");
  if (e != cudaSuccess) return fail(ctx, FLGF_ECUDA, std::string("refine_level: ") + cudaGetErrorString(e));
  return FLGF_OK;
}

// ----------------------------------------------------------------------------
// Read-only view of a context for other translation units of the library.
// ----------------------------------------------------------------------------
namespace flgf {
bool ctx_view(const flgf_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->N = c->N;
  v->fp64 = c->prec == FLGF_FP64;
  v->stream = c->stream;
  v->kspec = c->d_kspec;
  v->kstride = c->kstride;
  return true;
}
void ctx_set_error(flgf_ctx* c, const char* msg) {
  if (c) c->err = msg;
}
}  // namespace flgf
