// Host-only check of the dense MAC's parent-group packer (pack_parent_groups):
// on random block sets of every density, in both parent orders, every packed
// table must reproduce its parent records exactly -- targets, the neighbour
// cell of every (parent, e), the source block of every (cell, child) --
// every record must be packed exactly once, groups ordered by neighbour set
// must hold non-increasing set sizes, and every group must respect the
// thread, shared-memory and chunk limits of the kernel.
// Exit status 0 when every check passes.
#include <cstdio>
#include <map>
#include <random>
#include <vector>

#include "../../paper_1911_10228_gb300/csrc/internal.h"

using namespace flgf;

int main() {
  std::mt19937 rng(1);
  long total_bad = 0;
  for (int trial = 0; trial < 60; ++trial) {
    const int S = 4 + trial % 12;                     // box of S^3 blocks
    const double occ = 0.1 + 0.9 * (trial % 7) / 6.0;  // block density
    const bool excl = trial & 1;                       // level without near field
    const bool fp64 = trial % 3 == 0;
    std::vector<int> id(S * S * S, -1);
    int n = 0;
    for (auto& v : id)
      if (std::uniform_real_distribution<>(0, 1)(rng) < occ) v = n++;
    auto at = [&](int x, int y, int z) {
      return (x < 0 || y < 0 || z < 0 || x >= S || y >= S || z >= S) ? -1 : id[(x * S + y) * S + z];
    };
    std::vector<ParentRec> recs;
    for (int p0 = 0; p0 < S / 2; ++p0)
      for (int p1 = 0; p1 < S / 2; ++p1)
        for (int p2 = 0; p2 < S / 2; ++p2) {
          ParentRec r;
          bool has = false;
          for (int a = 0; a < 8; ++a) {
            r.tgt[a] = at(2 * p0 + (a >> 2), 2 * p1 + ((a >> 1) & 1), 2 * p2 + (a & 1));
            has |= r.tgt[a] >= 0;
          }
          if (!has) continue;
          for (int e = 0; e < 27; ++e)
            for (int b = 0; b < 8; ++b)
              r.cell[e][b] = excl && e == 13 ? -1
                                             : at(2 * (p0 + e / 9 - 1) + (b >> 2), 2 * (p1 + (e / 3) % 3 - 1) + ((b >> 1) & 1),
                                                  2 * (p2 + e % 3 - 1) + (b & 1));
          recs.push_back(r);
        }
    const int nchunk = 100;
    const bool by_list = (trial / 2) % 2 == 0;
    HadLists L;
    pack_parent_groups(trial % 3, recs, nchunk, had_kernel_units(fp64), L, by_list);
    // a record is identified by its first target
    std::map<int, size_t> rec_of;
    for (size_t i = 0; i < recs.size(); ++i)
      for (int t = 0; t < 8; ++t)
        if (recs[i].tgt[t] >= 0) { rec_of[recs[i].tgt[t]] = i; break; }
    std::vector<int> seen(recs.size(), 0);
    size_t m = 0;
    long bad = 0;
    for (const HadGroup& g : L.groups) {
      if (g.nact < 1 || g.nact > kHadMaxParents || g.pslots < g.nact || g.pslots * 2 * g.cpc > kHadThreads) ++bad;
      const size_t units = (size_t)(8 * g.ncell + had_kernel_units(fp64)) * g.cpc + (54 * g.nact + 31) / 32;
      if (32 * units > kHadSmemBytes || (int)units > L.max_units || g.ncell > 2047) ++bad;
      int prev_len = 27;
      for (int a = 0; a < g.nact; ++a, ++m) {
        int first = -1;
        for (int t = 0; t < 8 && first < 0; ++t) first = L.tgt_ids[g.tgt_off + a * 8 + t];
        if (!rec_of.count(first)) { ++bad; continue; }
        const size_t ri = rec_of[first];
        const ParentRec& r = recs[ri];
        seen[ri]++;
        if (!by_list) bad += ri != m;  // tile order keeps the record order
        for (int t = 0; t < 8; ++t) bad += L.tgt_ids[g.tgt_off + a * 8 + t] != r.tgt[t];
        int cell_of_e[27];
        int len = 0;
        for (int e = 0; e < 27; ++e) {
          const unsigned w = L.par_tab[g.par_off + e * g.nact + a];
          cell_of_e[e] = w == kNbEnd ? -1 : (int)w;
          if (cell_of_e[e] >= g.ncell) { ++bad; cell_of_e[e] = -1; }
          len += cell_of_e[e] >= 0;
        }
        if (by_list) bad += len > prev_len;
        prev_len = len;
        for (int e = 0; e < 27; ++e) {
          const int c = cell_of_e[e];
          bool any = false;
          for (int b = 0; b < 8; ++b) any |= r.cell[e][b] >= 0;
          if (any != (c >= 0)) { ++bad; continue; }
          for (int b = 0; b < 8; ++b) bad += (c >= 0 ? L.src_ids[g.src_off + b * g.ncell + c] : -1) != r.cell[e][b];
        }
      }
    }
    bad += m != recs.size();
    for (int v : seen) bad += v != 1;
    size_t covered = 0;
    for (const HadWork& w : L.work) {
      if (w.group < 0 || w.group >= (int)L.groups.size() || w.nch < 1 || w.nch > L.groups[w.group].cpc ||
          w.chunk0 < 0 || w.chunk0 + w.nch > nchunk)
        ++bad;
      covered += w.nch;
    }
    bad += covered != (size_t)nchunk * L.groups.size();
    if (bad) printf("trial %d: S=%d occupancy=%.2f parents=%zu groups=%zu: %ld mismatches\n", trial, S, occ,
                    recs.size(), L.groups.size(), bad);
    total_bad += bad;
  }
  printf("%s\n", total_bad ? "FAILED" : "ok");
  return total_bad ? 1 : 0;
}
