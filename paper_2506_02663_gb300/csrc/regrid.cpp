// Regridding (Sec. 5.4, RDM-2 and RDM-3): new level boxes from tagged cells by the clustering
// algorithm of Berger & Rigoutsos (signatures, holes, inflection points), built from the
// finest level down so that every new level nests in the next coarser one.  Host code; the
// tags come in as cell lists per level.
//
// Clustering of the tagged cells T of a region R (a box; the recursion partitions the level's
// domain into disjoint regions, each at least w cells wide in every dimension):
//   1. B = bounding box of T, widened inside R to at least w cells per dimension;
//   2. accept B when |T| >= efficiency * |B|;
//   3. otherwise cut B into two regions along one dimension, both at least w wide, at
//      (a) a hole: a cut next to an empty slice of the signature (tags per slice), the one
//          closest to the middle of its dimension; else
//      (b) an inflection point: a cut between slices whose second differences of the
//          signature have strictly opposite signs, the one with the largest jump; else
//      (c) the middle of the longest dimension that can be cut;
//      and recurse on the lower region, then the upper one; accept B when no cut is allowed.
//   Ties: the cut closest to its dimension's middle, then the longer dimension, then the
//   lower dimension, then the lower position.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "amr4_impl.h"

namespace amr4 {
namespace {

struct RBox {
  int lo[3];
  int hi[3];
};
using RBoxOut = RBox;

struct Cut {
  int d = -1;
  int c = 0;        // offset from the box's lo: the upper region starts at lo + c
  long long key[4];  // ordering key, smaller is better
};

bool better(const Cut& a, const Cut& b) {
  if (b.d < 0) return true;
  for (int i = 0; i < 4; ++i)
    if (a.key[i] != b.key[i]) return a.key[i] < b.key[i];
  return a.c < b.c;
}

class Clusterer {
 public:
  Clusterer(int D, double eff, int w) : D_(D), eff_(eff), w_(w) {}

  void run(std::vector<std::array<int, 3>>& tags, const RBox& region, std::vector<RBox>& out) {
    if (tags.empty()) return;
    RBox b{};
    for (int e = 0; e < 3; ++e) { b.lo[e] = 0; b.hi[e] = 0; }
    for (int e = 0; e < D_; ++e) {
      int lo = tags[0][e], hi = tags[0][e];
      for (const auto& t : tags) { lo = std::min(lo, t[e]); hi = std::max(hi, t[e]); }
      // widen to w cells inside the region: first upwards, then downwards
      int need = w_ - (hi - lo + 1);
      if (need > 0) {
        const int up = std::min(need, region.hi[e] - hi);
        hi += up;
        lo -= need - up;
      }
      b.lo[e] = lo;
      b.hi[e] = hi;
    }
    long long vol = 1;
    int n[3] = {1, 1, 1};
    for (int e = 0; e < D_; ++e) { n[e] = b.hi[e] - b.lo[e] + 1; vol *= n[e]; }
    if ((double)tags.size() >= eff_ * (double)vol) { out.push_back(b); return; }
    // signatures
    std::vector<long long> sig[3];
    for (int e = 0; e < D_; ++e) sig[e].assign(n[e], 0);
    for (const auto& t : tags)
      for (int e = 0; e < D_; ++e) ++sig[e][t[e] - b.lo[e]];
    Cut best;
    // (a) holes
    for (int e = 0; e < D_; ++e)
      for (int c = w_; c <= n[e] - w_; ++c)
        if (sig[e][c - 1] == 0 || sig[e][c] == 0) {
          Cut k;
          k.d = e;
          k.c = c;
          k.key[0] = 0;
          k.key[1] = std::llabs(2LL * c - n[e]);
          k.key[2] = -n[e];
          k.key[3] = e;
          if (better(k, best)) best = k;
        }
    // (b) inflection points
    if (best.d < 0)
      for (int e = 0; e < D_; ++e) {
        for (int c = std::max(w_, 2); c <= std::min(n[e] - w_, n[e] - 2); ++c) {
          const long long l0 = sig[e][c - 2] - 2 * sig[e][c - 1] + sig[e][c];
          const long long l1 = sig[e][c - 1] - 2 * sig[e][c] + sig[e][c + 1];
          if ((l0 < 0 && l1 > 0) || (l0 > 0 && l1 < 0)) {
            Cut k;
            k.d = e;
            k.c = c;
            k.key[0] = -std::llabs(l1 - l0);
            k.key[1] = std::llabs(2LL * c - n[e]);
            k.key[2] = -n[e];
            k.key[3] = e;
            if (better(k, best)) best = k;
          }
        }
      }
    // (c) bisection of the longest dimension that can be cut
    if (best.d < 0)
      for (int e = 0; e < D_; ++e)
        if (n[e] >= 2 * w_) {
          Cut k;
          k.d = e;
          k.c = n[e] / 2;
          k.key[0] = -n[e];
          k.key[1] = e;
          k.key[2] = 0;
          k.key[3] = 0;
          if (better(k, best)) best = k;
        }
    if (best.d < 0) { out.push_back(b); return; }
    RBox r0 = b, r1 = b;
    r0.hi[best.d] = b.lo[best.d] + best.c - 1;
    r1.lo[best.d] = b.lo[best.d] + best.c;
    std::vector<std::array<int, 3>> t0, t1;
    for (const auto& t : tags) (t[best.d] < r1.lo[best.d] ? t0 : t1).push_back(t);
    tags.clear();
    tags.shrink_to_fit();
    run(t0, r0, out);
    run(t1, r1, out);
  }

 private:
  int D_;
  double eff_;
  int w_;
};

amr_status regrid_boxes(int D, int r, const int* n0, int nlevels, const int* ntags, const int* const* tags,
                        double efficiency, int min_width, std::vector<std::vector<RBoxOut>>& levels,
                        std::string& err) {
  if (D != 2 && D != 3) { err = "regrid: dim must be 2 or 3"; return AMR_ERR_INVALID_ARG; }
  if (r != 2 && r != 4) { err = "regrid: ratio must be 2 or 4"; return AMR_ERR_INVALID_ARG; }
  if (nlevels < 1) { err = "regrid: nlevels must be >= 1"; return AMR_ERR_INVALID_ARG; }
  if (!(efficiency > 0.0 && efficiency <= 1.0)) { err = "regrid: efficiency must be in (0, 1]"; return AMR_ERR_INVALID_ARG; }
  const int wmin = (MIN_BOX + r - 1) / r;
  if (min_width < wmin) {
    err = "regrid: min_width must be at least " + std::to_string(wmin) + " (refined boxes need " +
          std::to_string(MIN_BOX) + " cells)";
    return AMR_ERR_INVALID_ARG;
  }
  for (int e = 0; e < D; ++e)
    if (n0[e] < min_width) {
      err = "regrid: min_width exceeds the level-0 extent";
      return AMR_ERR_INVALID_ARG;
    }
  const int grow = (NEST_MARGIN + r - 1) / r;  // coarse cells around coarsened finer boxes
  levels.assign(nlevels, {});
  // levels[l] for l >= 1: the new boxes of level l (level index space); levels[0] unused
  for (int l = nlevels - 2; l >= 0; --l) {
    long long nd[3] = {1, 1, 1};
    for (int e = 0; e < D; ++e) {
      nd[e] = n0[e];
      for (int q = 0; q < l; ++q) nd[e] *= r;
    }
    std::vector<long long> lin;
    auto push = [&](const int* c) {
      long long v = 0;
      for (int e = D - 1; e >= 0; --e) v = v * nd[e] + c[e];
      lin.push_back(v);
    };
    const int nt = ntags ? ntags[l] : 0;
    for (int i = 0; i < nt; ++i) {
      const int* c = tags[l] + (size_t)i * D;
      for (int e = 0; e < D; ++e)
        if (c[e] < 0 || c[e] >= nd[e]) {
          err = "regrid: tagged cell outside level " + std::to_string(l);
          return AMR_ERR_INVALID_ARG;
        }
      push(c);
    }
    if (l + 2 < nlevels)
      for (const RBoxOut& fb : levels[l + 2]) {
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int e = 0; e < D; ++e) {
          lo[e] = std::max(fb.lo[e] / (r * r) - grow, 0);
          hi[e] = (int)std::min<long long>(fb.hi[e] / (r * r) + grow, nd[e] - 1);
        }
        int c[3];
        for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
          for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
            for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) push(c);
      }
    std::sort(lin.begin(), lin.end());
    lin.erase(std::unique(lin.begin(), lin.end()), lin.end());
    std::vector<std::array<int, 3>> cells(lin.size());
    for (size_t i = 0; i < lin.size(); ++i) {
      long long v = lin[i];
      cells[i] = {0, 0, 0};
      for (int e = 0; e < D; ++e) { cells[i][e] = (int)(v % nd[e]); v /= nd[e]; }
    }
    RBox region{};
    for (int e = 0; e < 3; ++e) { region.lo[e] = 0; region.hi[e] = 0; }
    for (int e = 0; e < D; ++e) region.hi[e] = (int)nd[e] - 1;
    std::vector<RBox> out;
    Clusterer(D, efficiency, min_width).run(cells, region, out);
    for (const RBox& b : out) {
      RBoxOut f{};
      for (int e = 0; e < D; ++e) { f.lo[e] = b.lo[e] * r; f.hi[e] = (b.hi[e] + 1) * r - 1; }
      levels[l + 1].push_back(f);
    }
  }
  return AMR_OK;
}

}  // namespace
}  // namespace amr4

using namespace amr4;

amr_status amr_regrid(int dim, int ratio, const int* n0, int nlevels, const int* ntags, const int* const* tags,
                      const amr_regrid_params* p, int* new_nlevels, int* nboxes, int* boxes, int max_boxes) {
  if (!n0 || !p || (nlevels > 1 && ntags == nullptr)) {
    set_error("amr_regrid: null argument");
    return AMR_ERR_INVALID_ARG;
  }
  if (dim == 2 || dim == 3)
    for (int e = 0; e < dim; ++e)
      if (n0[e] < 1) {
        set_error("amr_regrid: n0 must be positive");
        return AMR_ERR_INVALID_ARG;
      }
  for (int l = 0; l + 1 < nlevels; ++l)
    if (ntags[l] < 0 || (ntags[l] > 0 && (tags == nullptr || tags[l] == nullptr))) {
      set_error("amr_regrid: tags of level " + std::to_string(l) + " missing");
      return AMR_ERR_INVALID_ARG;
    }
  std::vector<std::vector<RBoxOut>> lev;
  std::string err;
  const amr_status st = regrid_boxes(dim, ratio, n0, nlevels, ntags, tags, p->efficiency, p->min_width, lev, err);
  if (st != AMR_OK) {
    set_error(err);
    return st;
  }
  int nl = 1;
  while (nl < nlevels && !lev[nl].empty()) ++nl;
  long long total = 1;
  for (int l = 1; l < nl; ++l) total += (long long)lev[l].size();
  if (new_nlevels) *new_nlevels = nl;
  if (nboxes) {
    nboxes[0] = 1;
    for (int l = 1; l < nlevels; ++l) nboxes[l] = l < nl ? (int)lev[l].size() : 0;
  }
  if (boxes == nullptr) return AMR_OK;
  if (total > max_boxes) {
    set_error("amr_regrid: the new hierarchy has " + std::to_string(total) + " boxes, more than max_boxes (" +
              std::to_string(max_boxes) + ")");
    return AMR_ERR_INVALID_ARG;
  }
  int* q = boxes;
  for (int e = 0; e < dim; ++e) q[e] = 0;
  for (int e = 0; e < dim; ++e) q[dim + e] = n0[e] - 1;
  q += 2 * dim;
  for (int l = 1; l < nl; ++l)
    for (const RBoxOut& b : lev[l]) {
      for (int e = 0; e < dim; ++e) q[e] = b.lo[e];
      for (int e = 0; e < dim; ++e) q[dim + e] = b.hi[e];
      q += 2 * dim;
    }
  return AMR_OK;
}
