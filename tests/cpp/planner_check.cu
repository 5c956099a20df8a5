// Host-only check of the block-set planner: for meshes read from a file, every
// (target, source) interaction of every octree level must appear exactly once
// in the spectrum-MAC launch lists -- dense parent groups or pair lists -- with
// the kernel offset t - s, and every target exactly once, in a group of its
// own octree level.  The expected pairs are enumerated from the interaction
// rule directly: the children of the 27 neighbours of the target's parent that
// are sources, the near ones (|t - s|_inf <= 1) only on the finest octree
// level.  The forward phases and the adjoint phases (transposed leaf-only
// instances) are checked.  The planning runs on the CPU.
//
// usage: planner_check <mesh file> <list_pct> <t0> <t1> <t2> <fp64 0|1> [mac 0|1|2 [ncomp]]
// (mac: the FP32 spectrum-MAC form, FLGF_CTX_MAC: 1 = frequency-lane groups
// and frequency-lane pair lists, 2 = frequency-lane groups and shared-memory
// pair lists, 0 = parent groups and pair lists; FP64 always uses 0.  ncomp > 1: the
// problems are the components of a vector block set, whose identical meshes
// the file must hold; component 0's frequency-lane groups then stand for
// every component, at columns + c * cstride)
// mesh file (int32): N, n_problems, n_levels[n_problems], nblk[sum levels],
// coords[3 * sum nblk]
#include "../../paper_1911_10228_gb300/csrc/flgf_api.cu"

#include <cstdio>
#include <map>
#include <set>
#include <tuple>

int main(int argc, char** argv) {
  if (argc < 7 || argc > 9) {
    fprintf(stderr, "usage: %s mesh list_pct t0 t1 t2 fp64\n", argv[0]);
    return 2;
  }
  FILE* fp = fopen(argv[1], "rb");
  if (!fp) return 2;
  auto rd = [&](int* v, size_t n) { return fread(v, sizeof(int), n, fp) == n; };
  int N = 0, np = 0;
  if (!rd(&N, 1) || !rd(&np, 1)) return 2;
  std::vector<int> nlev(np);
  if (!rd(nlev.data(), np)) return 2;
  int nl = 0;
  for (int v : nlev) nl += v;
  std::vector<int> nblk(nl);
  if (!rd(nblk.data(), nl)) return 2;
  int nb = 0;
  for (int v : nblk) nb += v;
  std::vector<int32_t> coords(3 * (size_t)nb);
  if (!rd(coords.data(), coords.size())) return 2;
  fclose(fp);
  std::vector<double> h0(np, 1.0);

  flgf_ctx ctx;
  ctx.N = N;
  ctx.nI = 6;
  ctx.prec = atoi(argv[6]) ? FLGF_FP64 : FLGF_FP32;
  ctx.max_oct = 8;
  ctx.list_pct = atoi(argv[2]);
  ctx.mac = argc >= 8 ? atoi(argv[7]) : 1;
  for (int a = 0; a < 3; ++a) ctx.tile[a] = atoi(argv[3 + a]);
  auto bs = new flgf_blockset();
  bs->ctx = &ctx;
  bs->ncomp = argc == 9 ? atoi(argv[8]) : 1;
  const int rc = plan_blockset(&ctx, bs, np, nlev.data(), nblk.data(), coords.data(), h0.data());
  if (rc != FLGF_OK) {
    printf("plan failed (%d): %s\n", rc, ctx.err.c_str());
    return 1;
  }
  long bad = 0, pairs = 0, dense_pairs = 0, list_pairs = 0;
  // the launch lists of one phase (arena base) against the instances it serves
  auto check_phase = [&](const PhaseOff& ph, const char* base, const std::vector<const Inst*>& insts) {
    using Pair = std::tuple<int, int, int>;  // target, source (phase-local columns), offset index
    std::map<Pair, int> want, got;
    std::map<int, int> tlevel, written;      // target -> octree level, and times it is written
    for (const Inst* inp : insts) {
      const Inst& in = *inp;
      for (size_t k = 0; k < in.lv.size(); ++k)
        for (size_t i = 0; i < in.lv[k].size(); ++i) {
          if (!in.need_tgt[k][i]) continue;
          const int t = in.gid0[k] + (int)i - ph.gid_begin;
          tlevel[t] = (int)k;
          const I3& tc = in.lv[k][i];
          for (int e = 0; e < 27; ++e)
            for (int b = 0; b < 8; ++b) {
              const I3 sc = {2 * ((tc[0] >> 1) + e / 9 - 1) + (b >> 2), 2 * ((tc[1] >> 1) + (e / 3) % 3 - 1) + ((b >> 1) & 1),
                             2 * ((tc[2] >> 1) + e % 3 - 1) + (b & 1)};
              const int d0 = tc[0] - sc[0], d1 = tc[1] - sc[1], d2 = tc[2] - sc[2];
              if (k > 0 && std::abs(d0) <= 1 && std::abs(d1) <= 1 && std::abs(d2) <= 1) continue;
              auto it = in.idx[k].find(key3(sc));
              if (it == in.idx[k].end() || !in.is_src[k][it->second]) continue;
              want[Pair(t, in.gid0[k] + it->second - ph.gid_begin, off_index(d0, d1, d2))]++;
            }
        }
    }
    // dense parent groups
    const HadGroup* G = reinterpret_cast<const HadGroup*>(base + ph.hgroups);
    const int* src = reinterpret_cast<const int*>(base + ph.src_ids);
    const int* tgt = reinterpret_cast<const int*>(base + ph.tgt_ids);
    const uint16_t* par = reinterpret_cast<const uint16_t*>(base + ph.par_tab);
    for (int gi = 0; gi < ph.n_groups_dense; ++gi) {
      const HadGroup& g = G[gi];
      for (int m = 0; m < g.nact; ++m) {
        for (int a = 0; a < 8; ++a) {
          const int t = tgt[g.tgt_off + m * 8 + a];
          if (t < 0) continue;
          written[t]++;
          bad += tlevel.count(t) == 0 || tlevel[t] != g.level;
        }
        for (int e = 0; e < 27; ++e) {
          const unsigned w = par[g.par_off + e * g.nact + m];
          if (w == kNbEnd) continue;
          const int c = (int)w;
          if (c >= g.ncell) { ++bad; continue; }
          const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
          for (int b = 0; b < 8; ++b) {
            const int s = src[g.src_off + b * g.ncell + c];
            if (s < 0) continue;
            for (int a = 0; a < 8; ++a) {
              const int t = tgt[g.tgt_off + m * 8 + a];
              if (t < 0) continue;
              const int d0 = (a >> 2) - (b >> 2) - 2 * e0, d1 = ((a >> 1) & 1) - ((b >> 1) & 1) - 2 * e1,
                        d2 = (a & 1) - (b & 1) - 2 * e2;
              // near offsets above the finest octree level have zero kernel spectra
              if (g.level > 0 && std::abs(d0) <= 1 && std::abs(d1) <= 1 && std::abs(d2) <= 1) continue;
              got[Pair(t, s, off_index(d0, d1, d2))]++;
              ++dense_pairs;
            }
          }
        }
      }
    }
    // frequency-lane groups
    const FlGroup* FG = reinterpret_cast<const FlGroup*>(base + ph.fl_groups);
    const uint16_t* frows = reinterpret_cast<const uint16_t*>(base + ph.fl_rows);
    const uint32_t* fdlm = reinterpret_cast<const uint32_t*>(base + ph.fl_dlms);
    const int* ftgt0 = reinterpret_cast<const int*>(base + ph.fl_tgt);
    const int* fcells0 = reinterpret_cast<const int*>(base + ph.fl_cells);
    for (int gi = 0; gi < ph.n_fl; ++gi) {
      const FlGroup& g = FG[gi];
      bad += g.nact < 1 || g.nact > kFlMaxParents || g.nact > ph.fl_max_parents || g.ncell > kFlMaxCells ||
             g.ncell > ph.fl_max_cells;
      const int* ftgt = ftgt0 + (size_t)g.row_off * 8;
      const int* fcells = fcells0 + (size_t)g.cell_off * 8;
      for (int m = 0; m < g.nact; ++m) {
        for (int a = 0; a < 8; ++a) {
          const int t = ftgt[m * 8 + a];
          if (t < 0) continue;
          for (int c = 0; c < ph.fl_ncomp; ++c) {
            const int tc = t + c * ph.fl_cstride;
            written[tc]++;
            bad += tlevel.count(tc) == 0 || tlevel[tc] != g.level;
          }
        }
        const uint16_t* row = frows + (size_t)(g.row_off + m) * kFlRowStride;
        const int n = row[0];
        if (n > 27) { ++bad; continue; }
        int last_e = -1;
        for (int j = 0; j < n; ++j) {
          const int e = row[1 + j] >> 11, c = row[1 + j] & 0x7FF;
          if (e <= last_e || e > 26 || c >= g.ncell) { ++bad; continue; }
          last_e = e;
          const int e0 = e / 9 - 1, e1 = (e / 3) % 3 - 1, e2 = e % 3 - 1;
          // the delta mask: exactly the differences a - b of contributing pairs
          const uint32_t dword = fdlm[(size_t)(g.row_off + m) * kFlDelta + j];
          const uint32_t dmask = dword & ((1u << 27) - 1);
          uint32_t seen = 0;
          for (int b = 0; b < 8; ++b) {
            const int s = fcells[c * 8 + b];
            if (s < 0) continue;
            for (int a = 0; a < 8; ++a) {
              const int t = ftgt[m * 8 + a];
              if (t < 0) continue;
              const int d0 = (a >> 2) - (b >> 2) - 2 * e0, d1 = ((a >> 1) & 1) - ((b >> 1) & 1) - 2 * e1,
                        d2 = (a & 1) - (b & 1) - 2 * e2;
              if (g.level > 0 && std::abs(d0) <= 1 && std::abs(d1) <= 1 && std::abs(d2) <= 1) continue;
              const int dl = (((a >> 2) - (b >> 2) + 1) * 3 + (((a >> 1) & 1) - ((b >> 1) & 1) + 1)) * 3 +
                             ((a & 1) - (b & 1) + 1);
              seen |= 1u << dl;
              if (!((dmask >> dl) & 1u)) { ++bad; continue; }  // the kernel would skip this pair
              for (int cc = 0; cc < ph.fl_ncomp; ++cc)
                got[Pair(t + cc * ph.fl_cstride, s + cc * ph.fl_cstride, off_index(d0, d1, d2))]++;
              dense_pairs += ph.fl_ncomp;
            }
          }
          bad += seen != dmask;  // no delta without a product, and rows without products are dropped
          bad += (dword >> 27) != 0 && (dword >> 27) != 16;  // bits 27-30 clear
          if (dword >> 31) {  // a full row: every other delta is a near one of a coarse level
            for (int dl = 0; dl < 27; ++dl) {
              if ((dmask >> dl) & 1u) continue;
              const int d0 = dl / 9 - 1 - 2 * e0, d1 = (dl / 3) % 3 - 1 - 2 * e1, d2 = dl % 3 - 1 - 2 * e2;
              bad += !(g.level > 0 && std::abs(d0) <= 1 && std::abs(d1) <= 1 && std::abs(d2) <= 1);
            }
          }
        }
      }
    }
    // the product form of the phase: the two-path form exactly when at least
    // kFlSplitFullFraction of its rows are full
    {
      long rows = 0, full = 0;
      for (int gi = 0; gi < ph.n_fl; ++gi) {
        const FlGroup& g = FG[gi];
        for (int m = 0; m < g.nact; ++m) {
          const int n = frows[(size_t)(g.row_off + m) * kFlRowStride];
          rows += n;
          for (int j = 0; j < n; ++j) full += fdlm[(size_t)(g.row_off + m) * kFlDelta + j] >> 31;
        }
      }
      bad += ph.fl_split != (rows > 0 && (double)full >= kFlSplitFullFraction * (double)rows);
    }
    // frequency-lane pair lists
    const FllGroup* QG = reinterpret_cast<const FllGroup*>(base + ph.fll_groups);
    const int* qt = reinterpret_cast<const int*>(base + ph.fll_tgt);
    const int* qb = reinterpret_cast<const int*>(base + ph.fll_beg);
    const int* ql = reinterpret_cast<const int*>(base + ph.fll_len);
    const uint32_t* qe = reinterpret_cast<const uint32_t*>(base + ph.fll_ent);
    for (int gi = 0; gi < ph.n_fll; ++gi) {
      const FllGroup& g = QG[gi];
      bad += g.ntgt < 1 || g.ntgt > kFllTargets;
      for (int m = 0; m < g.ntgt; ++m) {
        const int i = g.tgt_off + m, t = qt[i];
        written[t]++;
        bad += tlevel.count(t) == 0 || tlevel[t] != g.level;
        bad += m > 0 && ql[i] > ql[i - 1];  // longest first
        for (int j = 0; j < ql[i]; ++j) {
          const uint32_t w = qe[qb[i] + j];
          got[Pair(t, (int)(w >> 9), (int)(w & 511))]++;
          ++list_pairs;
        }
      }
    }
    // pair lists
    const ListGroup* LG = reinterpret_cast<const ListGroup*>(base + ph.groups);
    const int* lt = reinterpret_cast<const int*>(base + ph.l_tgt);
    const int* ln = reinterpret_cast<const int*>(base + ph.l_len);
    const int* le = reinterpret_cast<const int*>(base + ph.l_ent);
    const int* ls = reinterpret_cast<const int*>(base + ph.l_src);
    for (int gi = 0; gi < ph.n_groups; ++gi) {
      const ListGroup& g = LG[gi];
      bad += g.ntgt < 1 || g.ntgt > kListTargets || g.nsrc > std::max(kListMaxSrc, 216);
      for (int m = 0; m < g.ntgt; ++m) {
        const int t = lt[g.tgt_off + m];
        written[t]++;
        bad += tlevel.count(t) == 0 || tlevel[t] != g.level;
        bad += ln[g.len_off + m] > g.maxlen;
        for (int j = 0; j < ln[g.len_off + m]; ++j) {
          const int w = le[g.ent_off + j * kListTargets + m];
          if ((w >> 9) >= g.nsrc) { ++bad; continue; }
          got[Pair(t, ls[g.src_off + (w >> 9)], w & 511)]++;
          ++list_pairs;
        }
      }
    }
    for (const auto& kv : tlevel) bad += written[kv.first] != 1;
    bad += written.size() != tlevel.size();
    for (const auto& kv : want) bad += kv.second != 1 || got[kv.first] != 1;
    bad += got.size() != want.size();
    pairs += (long)want.size();
  };
  for (int l = 0; l < bs->Lmax; ++l) {  // forward phases
    std::vector<const Inst*> insts;
    for (const Inst& in : bs->inst)
      if (in.l == l) insts.push_back(&in);
    check_phase(bs->ph[l], bs->ar.host.data(), insts);
  }
  // adjoint phases: build_adjoint compiles the transposed lists first and then
  // allocates device buffers, which fails without a GPU; the lists are complete
  build_adjoint(bs);
  for (int l = 0; l < bs->Lmax; ++l) {
    std::vector<const Inst*> insts;
    for (const Inst& in : bs->inst)
      if (in.l == l && in.variant == 0) insts.push_back(&in);
    for (const Inst& in : bs->adj_inst)
      if (in.l == l) insts.push_back(&in);
    if ((int)bs->aph.size() <= l) { ++bad; continue; }
    check_phase(bs->aph[l], bs->aar.host.data(), insts);
  }
  printf("pairs %ld (dense kernel %ld, pair lists %ld) mismatches %ld\n", pairs, dense_pairs, list_pairs, bad);
  printf("%s\n", bad ? "FAILED" : "ok");
  return bad ? 1 : 0;
}
