// Host side of libamr4: hierarchy validation (Eqs. grids, AMRHier, pBlock), composite
// field layout, index maps (Eq. validRegion, Fig. 1 (b)-(c)), and the device work lists for
// ghost filling (copy / AMRCFI, Sec. 5.2), refluxing (COH-3) and level transfers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <stdexcept>

#include <cuda_runtime.h>

#include "amr4_impl.h"

namespace amr4 {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* get_error() { return g_last_error.c_str(); }

// ------------------------------------------------------------------ exact rationals
namespace {
using i128 = __int128;
i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}
struct Q {
  i128 p = 0, q = 1;
  Q() = default;
  Q(i128 a, i128 b = 1) : p(a), q(b) { norm(); }
  void norm() {
    if (q < 0) { p = -p; q = -q; }
    i128 g = gcd128(p, q);
    if (g > 1) { p /= g; q /= g; }
  }
  Q operator+(const Q& o) const { return Q(p * o.q + o.p * q, q * o.q); }
  Q operator-(const Q& o) const { return Q(p * o.q - o.p * q, q * o.q); }
  Q operator*(const Q& o) const { return Q(p * o.p, q * o.q); }
  Q operator/(const Q& o) const { return Q(p * o.q, q * o.p); }
  bool zero() const { return p == 0; }
  double to_double() const { return static_cast<double>(static_cast<long long>(p)) / static_cast<double>(static_cast<long long>(q)); }
};
Q qpow(Q b, int e) {
  Q r(1);
  for (int i = 0; i < e; ++i) r = r * b;
  return r;
}
// int_lo^hi x^m dx
Q integ(Q lo, Q hi, int m) { return (qpow(hi, m + 1) - qpow(lo, m + 1)) / Q(m + 1); }
}  // namespace

// AMRCFI 1-D weights (Sec. 5.2 reading): the degree-4 polynomial whose averages over the
// 5 window cells [a, a+1] (a = 0..4) equal the coarse averages, averaged over fine
// sub-cell ``sub`` of window cell ``pos``.  w[(pos*r + sub)*5 + a].
void cfi_weights_exact(int r, std::vector<double>& w) {
  w.assign(CFI_W * r * CFI_W, 0.0);
  for (int pos = 0; pos < CFI_W; ++pos) {
    for (int sub = 0; sub < r; ++sub) {
      // solve M^T w = v, M[a][m] = int_a^{a+1} x^m, v[m] = r int_{pos+sub/r}^{pos+(sub+1)/r} x^m
      Q A[CFI_W][CFI_W + 1];
      for (int m = 0; m < CFI_W; ++m) {
        for (int a = 0; a < CFI_W; ++a) A[m][a] = integ(Q(a), Q(a + 1), m);
        A[m][CFI_W] = Q(r) * integ(Q(pos) + Q(sub, r), Q(pos) + Q(sub + 1, r), m);
      }
      for (int c = 0; c < CFI_W; ++c) {
        int piv = c;
        while (A[piv][c].zero()) ++piv;
        for (int k = 0; k <= CFI_W; ++k) std::swap(A[c][k], A[piv][k]);
        Q d = A[c][c];
        for (int k = 0; k <= CFI_W; ++k) A[c][k] = A[c][k] / d;
        for (int i = 0; i < CFI_W; ++i) {
          if (i == c || A[i][c].zero()) continue;
          Q f = A[i][c];
          for (int k = 0; k <= CFI_W; ++k) A[i][k] = A[i][k] - f * A[c][k];
        }
      }
      for (int a = 0; a < CFI_W; ++a) w[(pos * r + sub) * CFI_W + a] = A[a][CFI_W].to_double();
    }
  }
}

// ------------------------------------------------------------------ validation
static amr_status validate(const amr_hierarchy_desc* d, std::string& err) {
  const int D = d->dim;
  if (D != 2 && D != 3) { err = "dim must be 2 or 3"; return AMR_ERR_INVALID_ARG; }
  if (d->ratio != 2 && d->ratio != 4) { err = "ratio must be 2 or 4"; return AMR_ERR_INVALID_ARG; }
  for (int k = 0; k < D; ++k)
    if (d->n0[k] < 5) { err = "n0 must have >= 5 cells per dimension"; return AMR_ERR_INVALID_ARG; }
  if (!(d->h0 > 0.0)) { err = "h0 must be positive"; return AMR_ERR_INVALID_ARG; }
  if (d->nlevels < 1 || d->nboxes == nullptr || d->boxes == nullptr) { err = "no levels"; return AMR_ERR_INVALID_ARG; }
  if (d->nboxes[0] != 1) { err = "level 0 must be exactly one box"; return AMR_ERR_INVALID_ARG; }
  const int* b = d->boxes;
  for (int k = 0; k < D; ++k)
    if (b[k] != 0 || b[D + k] != d->n0[k] - 1) { err = "level 0 box must be the domain"; return AMR_ERR_INVALID_ARG; }
  const int r = d->ratio;
  // per box checks
  std::vector<std::vector<Box>> lv(d->nlevels);
  long long pos = 0;
  for (int l = 0; l < d->nlevels; ++l) {
    if (d->nboxes[l] < 1) { err = "empty level"; return AMR_ERR_INVALID_ARG; }
    long long scale = 1;
    for (int i = 0; i < l; ++i) scale *= r;
    for (int k = 0; k < d->nboxes[l]; ++k) {
      Box bx{};
      for (int e = 0; e < 3; ++e) { bx.lo[e] = 0; bx.hi[e] = 0; }
      for (int e = 0; e < D; ++e) { bx.lo[e] = d->boxes[pos + e]; bx.hi[e] = d->boxes[pos + D + e]; }
      pos += 2 * D;
      lv[l].push_back(bx);
      if (l == 0) continue;
      for (int e = 0; e < D; ++e) {
        long long nd = d->n0[e] * scale;
        if (bx.lo[e] > bx.hi[e] || bx.lo[e] < 0 || bx.hi[e] >= nd) {
          err = "box " + std::to_string(k) + " of level " + std::to_string(l) + " out of bounds";
          return AMR_ERR_INVALID_ARG;
        }
      }
      for (int e = 0; e < D; ++e)
        if (bx.hi[e] - bx.lo[e] + 1 < MIN_BOX) {
          err = "box " + std::to_string(k) + " of level " + std::to_string(l) + " smaller than 4";
          return AMR_ERR_BOX_TOO_SMALL;
        }
      for (int e = 0; e < D; ++e)
        if (bx.lo[e] % r != 0 || (bx.hi[e] + 1) % r != 0) {
          err = "box " + std::to_string(k) + " of level " + std::to_string(l) + " not properly refined";
          return AMR_ERR_REFINEMENT;
        }
    }
  }
  for (int l = 1; l < d->nlevels; ++l) {
    for (size_t i = 0; i < lv[l].size(); ++i)
      for (size_t j = i + 1; j < lv[l].size(); ++j) {
        bool ov = true;
        for (int e = 0; e < D; ++e)
          ov = ov && std::max(lv[l][i].lo[e], lv[l][j].lo[e]) <= std::min(lv[l][i].hi[e], lv[l][j].hi[e]);
        if (ov) { err = "boxes overlap on level " + std::to_string(l); return AMR_ERR_INVALID_ARG; }
      }
  }
  for (int l = 2; l < d->nlevels; ++l) {
    long long nc[3] = {1, 1, 1};
    long long scale = 1;
    for (int i = 0; i < l - 1; ++i) scale *= r;
    for (int e = 0; e < D; ++e) nc[e] = d->n0[e] * scale;
    for (size_t k = 0; k < lv[l].size(); ++k) {
      int glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
      for (int e = 0; e < D; ++e) {
        glo[e] = std::max(lv[l][k].lo[e] / r - NEST_MARGIN, 0);
        ghi[e] = (int)std::min<long long>(lv[l][k].hi[e] / r + NEST_MARGIN, nc[e] - 1);
      }
      // the grown region must be covered by the union of level l-1 boxes: count cells
      long long need = 1, have = 0;
      for (int e = 0; e < D; ++e) need *= (ghi[e] - glo[e] + 1);
      for (const Box& c : lv[l - 1]) {
        long long v = 1;
        for (int e = 0; e < D; ++e) {
          int a = std::max(glo[e], c.lo[e]), bb = std::min(ghi[e], c.hi[e]);
          v *= (bb >= a) ? (bb - a + 1) : 0;
        }
        have += v;  // level l-1 boxes are disjoint
      }
      if (have != need) {
        err = "box " + std::to_string(k) + " of level " + std::to_string(l) + " not properly nested";
        return AMR_ERR_NESTING;
      }
    }
  }
  // coarsest level-0 multigrid grid
  int n[3] = {1, 1, 1};
  for (int e = 0; e < D; ++e) n[e] = d->n0[e];
  for (;;) {
    bool ok = true;
    for (int e = 0; e < D; ++e) ok = ok && (n[e] % 2 == 0) && (n[e] / 2 >= MIN_BOX);
    if (!ok) break;
    for (int e = 0; e < D; ++e) n[e] /= 2;
  }
  long long cells = 1;
  for (int e = 0; e < D; ++e) cells *= n[e];
  if (cells > MAX_BOTTOM) { err = "coarsest multigrid grid too large for the dense bottom solve"; return AMR_ERR_INVALID_ARG; }
  return AMR_OK;
}

// ------------------------------------------------------------------ helpers
static PatchDesc make_patch(const int n[3], const int lo[3], int D, long long& cursor) {
  PatchDesc p{};
  const long long px = ((n[0] + 2 * NG) + 3) / 4 * 4;  // x pitch, multiple of 4 elements
  p.sy = px;
  p.sz = (D == 3) ? px * (n[1] + 2 * NG) : 0;
  for (int e = 0; e < 3; ++e) { p.n[e] = n[e]; p.lo[e] = lo[e]; }
  const long long total = (D == 3) ? p.sz * (n[2] + 2 * NG) : p.sy * (n[1] + 2 * NG);
  cursor = (cursor + 31) / 32 * 32;  // 256-byte aligned patches (FP64)
  p.off = cursor;
  cursor += total;
  return p;
}

static inline long long cell_off(const PatchDesc& p, int D, int i, int j, int k) {
  return p.off + (long long)(i + NG) + (long long)(j + NG) * p.sy + (D == 3 ? (long long)(k + NG) * p.sz : 0);
}

template <typename T>
static T* upload(const std::vector<T>& v) {
  if (v.empty()) return nullptr;
  T* d = nullptr;
  if (cudaMalloc(&d, v.size() * sizeof(T)) != cudaSuccess) throw std::runtime_error("cudaMalloc failed");
  if (cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    throw std::runtime_error("cudaMemcpy failed");
  return d;
}

// CF ghosts grouped by coarse parent (entries with one key): the shared window (origin,
// coarse patch, position) of the first child, each child's destination at index sub_x +
// 2 sub_y + 4 sub_z.  Ratio 2 only (no groups otherwise: the per-ghost list is used).
// Orders a level's interface faces by connected component (stable within a component) and
// records the component ranges; on entry cic_comp holds each face's patch index.
static void group_cic_faces(LevelHost& L, const std::vector<int>& im_component, int D) {
  const size_t nb = L.boxes.size();
  std::vector<int> label(nb), comp_of_label(nb, -1);
  for (size_t k = 0; k < nb; ++k) label[k] = im_component[L.first_patch + k];
  int ncomp = 0;
  for (size_t k = 0; k < nb; ++k)  // labels are the smallest box index of each component
    if (label[k] == (int)k) comp_of_label[k] = ncomp++;
  const size_t nf = L.cicf.size();
  std::vector<int> comp(nf);
  for (size_t i = 0; i < nf; ++i) comp[i] = comp_of_label[label[L.cic_comp[i]]];
  std::vector<size_t> ord(nf);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return comp[a] < comp[b]; });
  std::vector<CicFace> f(nf);
  std::vector<int> cell(nf * D), cc(nf);
  for (size_t i = 0; i < nf; ++i) {
    f[i] = L.cicf[ord[i]];
    cc[i] = comp[ord[i]];
    for (int e = 0; e < D; ++e) cell[i * D + e] = L.cic_cell[ord[i] * D + e];
  }
  L.cicf.swap(f);
  L.cic_cell.swap(cell);
  L.cic_comp.swap(cc);
  L.cic_cstart.assign(ncomp + 1, 0);
  for (size_t i = 0; i < nf; ++i) ++L.cic_cstart[L.cic_comp[i] + 1];
  for (int c = 0; c < ncomp; ++c) L.cic_cstart[c + 1] += L.cic_cstart[c];
  // single-box components: per face the slot of its box problem's boundary data (faces f =
  // 2d + side in order, each over the box's cells with dimension d removed, lowest remaining
  // dimension fastest)
  std::vector<int> nbox(ncomp, 0), onebox(ncomp, -1);
  for (size_t k = 0; k < nb; ++k) {
    const int c = comp_of_label[label[k]];
    ++nbox[c];
    onebox[c] = (int)k;
  }
  L.cic_comp_box.assign(ncomp, -1);
  for (int c = 0; c < ncomp; ++c)
    if (nbox[c] == 1) L.cic_comp_box[c] = onebox[c];
  L.cic_slot.assign(nf, -1);
  for (size_t i = 0; i < nf; ++i) {
    const int b = L.cic_comp_box[L.cic_comp[i]];
    if (b < 0) continue;
    const Box& B = L.boxes[b];
    int n[3] = {1, 1, 1};
    for (int e = 0; e < D; ++e) n[e] = B.hi[e] - B.lo[e] + 1;
    const int d = L.cicf[i].dir, f = 2 * d + (L.cicf[i].side > 0 ? 1 : 0);
    long long off = 0;
    for (int f2 = 0; f2 < f; ++f2) {
      long long cnt = 1;
      for (int e = 0; e < D; ++e)
        if (e != f2 / 2) cnt *= n[e];
      off += cnt;
    }
    long long idx = 0, stride = 1;
    for (int e = 0; e < D; ++e) {
      if (e == d) continue;
      idx += (long long)(L.cic_cell[i * D + e] - B.lo[e]) * stride;
      stride *= n[e];
    }
    L.cic_slot[i] = off + idx;
  }
  // chunks of at most CIC_CHUNK faces, at least one (possibly empty) per component
  constexpr int CIC_CHUNK = 2048;
  L.cic_chunks.clear();
  L.cic_ccstart.assign(1, 0);
  for (int c = 0; c < ncomp; ++c) {
    const int b = L.cic_cstart[c], e = L.cic_cstart[c + 1];
    int q = b;
    do {
      const int qe = std::min(e, q + CIC_CHUNK);
      L.cic_chunks.push_back({c, q, qe, 0});
      q = qe;
    } while (q < e);
    L.cic_ccstart.push_back((int)L.cic_chunks.size());
  }
}

static std::vector<CfiGroup> cfi_groups(const std::vector<CfiEntry>& cfi, const std::vector<long long>& key, int r,
                                        int D) {
  std::vector<CfiGroup> out;
  if (r != 2 || cfi.empty() || key.size() != cfi.size()) return out;
  std::vector<size_t> ord(cfi.size());
  std::iota(ord.begin(), ord.end(), size_t(0));
  std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return key[a] < key[b]; });
  for (size_t i = 0; i < ord.size();) {
    const CfiEntry& e0 = cfi[ord[i]];
    CfiGroup g{};
    g.src = e0.src;
    g.cpatch = e0.cpatch;
    for (int e = 0; e < 3; ++e) g.pos[e] = e0.pos[e];
    for (int c = 0; c < 8; ++c) g.dst[c] = -1;
    size_t j = i;
    for (; j < ord.size() && key[ord[j]] == key[ord[i]]; ++j) {
      const CfiEntry& e = cfi[ord[j]];
      const int c = e.sub[0] + 2 * e.sub[1] + (D == 3 ? 4 * e.sub[2] : 0);
      g.dst[c] = e.dst;
    }
    out.push_back(g);
    i = j;
  }
  return out;
}

namespace {
// level lookup over the level's bounding box (+ margin): patch id per cell, -1 outside
struct LevelMap {
  int D = 2, lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
  std::vector<int> pid;
  void build(const std::vector<Box>& boxes, int D_) {
    D = D_;
    for (int e = 0; e < 3; ++e) { lo[e] = 0; ext[e] = 1; }
    for (int e = 0; e < D; ++e) {
      int a = boxes[0].lo[e], b = boxes[0].hi[e];
      for (const Box& bx : boxes) { a = std::min(a, bx.lo[e]); b = std::max(b, bx.hi[e]); }
      lo[e] = a;
      ext[e] = b - a + 1;
    }
    pid.assign((size_t)ext[0] * ext[1] * ext[2], -1);
    for (size_t k = 0; k < boxes.size(); ++k) {
      const Box& bx = boxes[k];
      for (int z = (D == 3 ? bx.lo[2] : 0); z <= (D == 3 ? bx.hi[2] : 0); ++z)
        for (int y = bx.lo[1]; y <= bx.hi[1]; ++y)
          for (int x = bx.lo[0]; x <= bx.hi[0]; ++x) pid[idx(x, y, z)] = (int)k;
    }
  }
  size_t idx(int x, int y, int z) const {
    return ((size_t)(z - lo[2]) * ext[1] + (size_t)(y - lo[1])) * ext[0] + (size_t)(x - lo[0]);
  }
  int at(const int g[3]) const {
    for (int e = 0; e < D; ++e)
      if (g[e] < lo[e] || g[e] >= lo[e] + ext[e]) return -1;
    return pid[idx(g[0], g[1], D == 3 ? g[2] : 0)];
  }
};
}  // namespace

// ------------------------------------------------------------------ build
amr_status build_hierarchy(const amr_hierarchy_desc* desc, amr_hierarchy* h, std::string& err) {
  amr_status st = validate(desc, err);
  if (st != AMR_OK) return st;
  const int D = desc->dim, r = desc->ratio;
  h->D = D;
  h->r = r;
  h->L = desc->nlevels;
  h->h0 = desc->h0;
  for (int e = 0; e < 3; ++e) h->n0[e] = (e < D) ? desc->n0[e] : 1;
  h->lev.resize(h->L);
  long long cursor = 0, pos = 0;
  int gp = 0;
  for (int l = 0; l < h->L; ++l) {
    LevelHost& L = h->lev[l];
    long long scale = 1;
    for (int i = 0; i < l; ++i) scale *= r;
    for (int e = 0; e < 3; ++e) L.ndom[e] = (e < D) ? (int)(h->n0[e] * scale) : 1;
    L.h = h->h0 / (double)scale;
    L.first_patch = gp;
    for (int k = 0; k < desc->nboxes[l]; ++k) {
      Box bx{};
      for (int e = 0; e < D; ++e) { bx.lo[e] = desc->boxes[pos + e]; bx.hi[e] = desc->boxes[pos + D + e]; }
      pos += 2 * D;
      L.boxes.push_back(bx);
      int n[3] = {1, 1, 1}, lo[3] = {0, 0, 0};
      for (int e = 0; e < D; ++e) { n[e] = bx.hi[e] - bx.lo[e] + 1; lo[e] = bx.lo[e]; }
      PatchDesc p = make_patch(n, lo, D, cursor);
      L.patches.push_back(p);
      for (int e = 0; e < 3; ++e) L.maxn[e] = std::max(L.maxn[e], n[e]);
      amr_patch_info pi{};
      pi.level = l;
      pi.box = k;
      for (int e = 0; e < 3; ++e) { pi.lo[e] = (e < D) ? bx.lo[e] : 0; pi.hi[e] = (e < D) ? bx.hi[e] : 0; }
      pi.offset = p.off;
      pi.stride_y = p.sy;
      pi.stride_z = p.sz;
      pi.nelems = (D == 3) ? p.sz * (n[2] + 2 * NG) : p.sy * (n[1] + 2 * NG);
      h->pinfo.push_back(pi);
      ++gp;
    }
  }
  h->nelems = (cursor + 31) / 32 * 32;
  h->npatch = gp;

  std::vector<LevelMap> maps(h->L);
  for (int l = 0; l < h->L; ++l) maps[l].build(h->lev[l].boxes, D);

  // ---- valid mask (Eq. validRegion) ----
  for (int l = 0; l < h->L; ++l) {
    LevelHost& L = h->lev[l];
    for (size_t k = 0; k < L.boxes.size(); ++k) {
      const PatchDesc& p = L.patches[k];
      for (int z = 0; z < p.n[2]; ++z)
        for (int y = 0; y < p.n[1]; ++y)
          for (int x = 0; x < p.n[0]; ++x) {
            int g[3] = {p.lo[0] + x, p.lo[1] + y, p.lo[2] + z};
            bool v = true;
            if (l + 1 < h->L) {
              int f[3] = {g[0] * r, g[1] * r, D == 3 ? g[2] * r : 0};
              v = maps[l + 1].at(f) < 0;
            }
            h->im_valid.push_back(v ? 1 : 0);
          }
    }
  }

  // ---- connected components per level (union-find over face adjacency) ----
  for (int l = 0; l < h->L; ++l) {
    const auto& B = h->lev[l].boxes;
    std::vector<int> parent(B.size());
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int i) { while (parent[i] != i) i = parent[i]; return i; };
    for (size_t i = 0; i < B.size(); ++i)
      for (size_t j = i + 1; j < B.size(); ++j) {
        bool adj = false;
        for (int d = 0; d < D && !adj; ++d) {
          bool touch = (B[i].hi[d] + 1 == B[j].lo[d]) || (B[j].hi[d] + 1 == B[i].lo[d]);
          if (!touch) continue;
          bool ov = true;
          for (int e = 0; e < D; ++e)
            if (e != d) ov = ov && std::max(B[i].lo[e], B[j].lo[e]) <= std::min(B[i].hi[e], B[j].hi[e]);
          adj = ov;
        }
        if (adj) {
          int a = find((int)i), b = find((int)j);
          parent[std::max(a, b)] = std::min(a, b);
        }
      }
    for (size_t i = 0; i < B.size(); ++i) h->im_component.push_back(find((int)i));
  }

  // ---- ghost maps, copy lists, AMRCFI lists ----
  cfi_weights_exact(r, h->cfi_w);
  long long padded_base = 0;
  for (int l = 0; l < h->L; ++l) {
    LevelHost& L = h->lev[l];
    for (size_t k = 0; k < L.boxes.size(); ++k) {
      const PatchDesc& p = L.patches[k];
      int ext[3] = {1, 1, 1};
      for (int e = 0; e < D; ++e) ext[e] = p.n[e] + 2 * NG;
      long long cidx = 0;
      for (int az = 0; az < ext[2]; ++az)
        for (int ay = 0; ay < ext[1]; ++ay)
          for (int ax = 0; ax < ext[0]; ++ax, ++cidx) {
            int a[3] = {ax, ay, az};
            int g[3] = {0, 0, 0};
            int nout = 0, dout = -1;
            for (int e = 0; e < D; ++e) {
              g[e] = p.lo[e] - NG + a[e];
              if (g[e] < p.lo[e] || g[e] > p.lo[e] + p.n[e] - 1) { ++nout; dout = e; }
            }
            int code = 4, src = -1, aux = -1;
            if (nout == 0) {
              code = 0;
            } else if (nout == 1) {
              const int d = dout;
              if (g[d] < 0 || g[d] >= L.ndom[d]) {
                code = 1;
                const int side = g[d] < 0 ? 0 : 1;
                src = 2 * d + side;
                aux = side == 0 ? -g[d] : g[d] - L.ndom[d] + 1;
              } else {
                int q = maps[l].at(g);
                if (q >= 0 && q != (int)k) {
                  code = 2;
                  src = q;
                  const PatchDesc& s = L.patches[q];
                  long long lin = 0, stride = 1;
                  for (int e = 0; e < D; ++e) { lin += (g[e] - s.lo[e]) * stride; stride *= s.n[e]; }
                  aux = (int)lin;
                  int sx = g[0] - s.lo[0], sy = g[1] - s.lo[1], sz = D == 3 ? g[2] - s.lo[2] : 0;
                  L.copy.push_back({p.off + (long long)ax + (long long)ay * p.sy + (long long)az * p.sz,
                                    cell_off(s, D, sx, sy, sz)});
                } else {
                  code = 3;
                  // AMRCFI entry (level >= 1 by construction: level 0 is the domain)
                  const LevelHost& C = h->lev[l - 1];
                  CfiEntry ce{};
                  ce.dst = p.off + (long long)ax + (long long)ay * p.sy + (long long)az * p.sz;
                  ce.dir = (signed char)d;
                  ce.layer = (signed char)(g[d] < p.lo[d] ? -(p.lo[d] - g[d]) : (g[d] - (p.lo[d] + p.n[d] - 1)));
                  ce.fpatch = (int)k;
                  int start[3] = {0, 0, 0};
                  for (int e = 0; e < 3; ++e) { ce.pos[e] = 0; ce.sub[e] = 0; }
                  for (int e = 0; e < D; ++e) {
                    int par = (int)std::floor((double)g[e] / r);
                    int s0 = std::min(std::max(par - 2, 0), C.ndom[e] - CFI_W);
                    start[e] = s0;
                    ce.pos[e] = (signed char)(par - s0);
                    ce.sub[e] = (signed char)(g[e] - r * par);
                  }
                  // window inside one coarse patch?
                  int cp0 = maps[l - 1].at(start);
                  int endc[3] = {start[0] + CFI_W - 1, start[1] + CFI_W - 1, D == 3 ? start[2] + CFI_W - 1 : 0};
                  bool single = cp0 >= 0;
                  if (single) {
                    const PatchDesc& cpd = C.patches[cp0];
                    for (int e = 0; e < D; ++e)
                      single = single && endc[e] <= cpd.lo[e] + cpd.n[e] - 1 && start[e] >= cpd.lo[e];
                  }
                  if (single) {
                    const PatchDesc& cpd = C.patches[cp0];
                    ce.cpatch = cp0;
                    ce.src = cell_off(cpd, D, start[0] - cpd.lo[0], start[1] - cpd.lo[1], D == 3 ? start[2] - cpd.lo[2] : 0);
                  } else {
                    ce.cpatch = -1;
                    ce.src = -1 - (long long)(L.cfi_side.size() / (D == 3 ? 125 : 25));
                    for (int wz = 0; wz < (D == 3 ? CFI_W : 1); ++wz)
                      for (int wy = 0; wy < CFI_W; ++wy)
                        for (int wx = 0; wx < CFI_W; ++wx) {
                          int c[3] = {start[0] + wx, start[1] + wy, D == 3 ? start[2] + wz : 0};
                          int q2 = maps[l - 1].at(c);
                          if (q2 < 0) { err = "AMRCFI window leaves level " + std::to_string(l - 1); return AMR_ERR_NESTING; }
                          const PatchDesc& cpd = C.patches[q2];
                          L.cfi_side.push_back(cell_off(cpd, D, c[0] - cpd.lo[0], c[1] - cpd.lo[1], D == 3 ? c[2] - cpd.lo[2] : 0));
                        }
                  }
                  L.cfi.push_back(ce);
                  if (ce.layer == 1 || ce.layer == -1) {  // a coarse-fine interface face
                    const long long stride = d == 0 ? 1 : (d == 1 ? p.sy : p.sz);
                    L.cicf.push_back({ce.dst, ce.layer * stride, d, (int)ce.layer});
                    for (int e = 0; e < D; ++e) L.cic_cell.push_back(e == d ? g[e] - ce.layer : g[e]);
                    L.cic_comp.push_back((int)k);  // patch for now; component below
                  }
                  {
                    // grouping key: fine patch, face, coarse parent
                    long long key = (long long)k * 6 + 2 * d + (g[d] < p.lo[d] ? 0 : 1);
                    for (int e = D - 1; e >= 0; --e) key = key * C.ndom[e] + (long long)std::floor((double)g[e] / r);
                    L.cfi_key.push_back(key);
                  }
                  h->im_cfi_cell.push_back(padded_base + cidx);
                  for (int e = 0; e < D; ++e) {
                    h->im_cfi_start.push_back(start[e]);
                    h->im_cfi_pos.push_back(ce.pos[e]);
                    h->im_cfi_sub.push_back(ce.sub[e]);
                  }
                }
              }
            }
            h->im_code.push_back(code);
            h->im_src.push_back(src);
            h->im_aux.push_back(aux);
          }
      padded_base += cidx;
    }
    group_cic_faces(L, h->im_component, D);
  }

  // ---- reflux lists (COH-3) and transfer blocks ----
  for (int l = 0; l + 1 < h->L; ++l) {
    LevelHost& L = h->lev[l];
    const LevelHost& F = h->lev[l + 1];
    // coarse map of the fine level's coarsened boxes
    std::vector<Box> cb;
    for (const Box& fb : F.boxes) {
      Box c{};
      for (int e = 0; e < 3; ++e) { c.lo[e] = 0; c.hi[e] = 0; }
      for (int e = 0; e < D; ++e) { c.lo[e] = fb.lo[e] / r; c.hi[e] = fb.hi[e] / r; }
      cb.push_back(c);
    }
    LevelMap fm;
    fm.build(cb, D);
    for (size_t k = 0; k < L.boxes.size(); ++k) {
      const PatchDesc& p = L.patches[k];
      long long lin = 0;
      for (int z = 0; z < p.n[2]; ++z)
        for (int y = 0; y < p.n[1]; ++y)
          for (int x = 0; x < p.n[0]; ++x, ++lin) {
            int g[3] = {p.lo[0] + x, p.lo[1] + y, p.lo[2] + z};
            if (fm.at(g) >= 0) continue;  // invalid cell
            RefluxEntry re{};
            re.faces = 0;
            for (int f = 0; f < 6; ++f) re.fpatch[f] = -1;
            for (int d = 0; d < D; ++d)
              for (int side = 0; side < 2; ++side) {
                int nb[3] = {g[0], g[1], g[2]};
                nb[d] += side ? 1 : -1;
                if (nb[d] < 0 || nb[d] >= L.ndom[d]) continue;
                int fp = fm.at(nb);
                if (fp >= 0) {
                  re.faces |= 1 << (2 * d + side);
                  re.fpatch[2 * d + side] = fp;
                }
              }
            if (re.faces == 0) continue;
            re.coff = cell_off(p, D, x, y, z);
            re.cpatch = (int)k;
            for (int e = 0; e < 3; ++e) re.g[e] = g[e];
            L.reflux.push_back(re);
            h->im_reflux_cell.push_back(l);
            h->im_reflux_cell.push_back((int)k);
            h->im_reflux_cell.push_back((int)lin);
            h->im_reflux_faces.push_back(re.faces);
          }
    }
    for (size_t fk = 0; fk < F.boxes.size(); ++fk)
      for (size_t ck = 0; ck < L.boxes.size(); ++ck) {
        XferBlock xb{};
        xb.fpatch = (int)fk;
        xb.cpatch = (int)ck;
        bool any = true;
        for (int e = 0; e < 3; ++e) { xb.clo[e] = 0; xb.chi[e] = 0; }
        for (int e = 0; e < D; ++e) {
          xb.clo[e] = std::max(cb[fk].lo[e], L.boxes[ck].lo[e]);
          xb.chi[e] = std::min(cb[fk].hi[e], L.boxes[ck].hi[e]);
          any = any && xb.chi[e] >= xb.clo[e];
        }
        if (!any) continue;
        L.xfer.push_back(xb);
        for (int e = 0; e < D; ++e) L.dev.xfer_max[e] = std::max(L.dev.xfer_max[e], xb.chi[e] - xb.clo[e] + 1);
      }
  }

  // ---- boundary-data layout ----
  h->bc_off.assign((size_t)h->L * 2 * D + 1, 0);
  long long bcur = 0;
  for (int l = 0; l < h->L; ++l)
    for (int f = 0; f < 2 * D; ++f) {
      h->bc_off[(size_t)l * 2 * D + f] = bcur;
      long long cnt = 1;
      for (int e = 0; e < D; ++e)
        if (e != f / 2) cnt *= h->lev[l].ndom[e];
      bcur += cnt;
    }
  h->bc_off[(size_t)h->L * 2 * D] = bcur;

  // ---- level-0 multigrid pyramid ----
  {
    int n[3] = {h->n0[0], h->n0[1], h->n0[2]};
    double hh = h->h0;
    for (;;) {
      MgGrid g;
      for (int e = 0; e < 3; ++e) g.n[e] = n[e];
      g.h = hh;
      long long c = 0;
      int lo[3] = {0, 0, 0};
      g.patch = make_patch(n, lo, D, c);
      g.patch.off = 0;
      g.nelems = (c + 31) / 32 * 32;
      h->mg.push_back(g);
      bool ok = true;
      for (int e = 0; e < D; ++e) ok = ok && (n[e] % 2 == 0) && (n[e] / 2 >= MIN_BOX);
      if (!ok) break;
      for (int e = 0; e < D; ++e) n[e] /= 2;
      hh *= 2.0;
    }
  }

  return AMR_OK;
}

// Replicas of a hierarchy for stacked component batches: every field of the stacked
// hierarchy is k copies of h's composite layout, copy c at element offset c * stride.  Patch
// indices inside the work lists (AMRCFI source patches, refluxing and transfer patch pairs)
// are indices within a level, so replica c shifts them by c times the level's patch count;
// element offsets shift by c * stride.  The level-0 multigrid grids keep one layout each and
// get k replicas at their own stride.
amr_status stack_hierarchy(const amr_hierarchy* h, int k, amr_hierarchy** out, std::string& err) {
  if (k < 1 || h->ncomp != 1) {
    err = "stack_hierarchy: needs k >= 1 and an unstacked hierarchy";
    return AMR_ERR_INVALID_ARG;
  }
  std::unique_ptr<amr_hierarchy> s(new amr_hierarchy());
  s->D = h->D;
  s->r = h->r;
  for (int e = 0; e < 3; ++e) s->n0[e] = h->n0[e];
  s->h0 = h->h0;
  s->L = h->L;
  s->ncomp = k;
  const long long stride = (h->nelems + 63) / 64 * 64;
  s->cstride = stride;
  s->nelems = stride * k;
  s->npatch = h->npatch * k;
  s->bc_off = h->bc_off;
  s->cfi_w = h->cfi_w;
  s->lev.resize(h->L);
  for (int l = 0; l < h->L; ++l) {
    const LevelHost& A = h->lev[l];
    LevelHost& B = s->lev[l];
    const int np = (int)A.patches.size();
    const int npc = l > 0 ? (int)h->lev[l - 1].patches.size() : 0;  // coarse level's patches
    const int npf = l + 1 < h->L ? (int)h->lev[l + 1].patches.size() : 0;
    for (int e = 0; e < 3; ++e) { B.ndom[e] = A.ndom[e]; B.maxn[e] = A.maxn[e]; }
    B.h = A.h;
    B.first_patch = A.first_patch * k;
    const long long w3 = h->D == 3 ? 125 : 25;
    const long long nside = (long long)A.cfi_side.size() / w3;
    long long key_span = 1;  // replica c's grouping keys are shifted by c * key_span
    for (long long key : A.cfi_key) key_span = std::max(key_span, key + 1);
    for (int c = 0; c < k; ++c) {
      const long long o = c * stride;
      for (const Box& b : A.boxes) B.boxes.push_back(b);
      for (PatchDesc p : A.patches) {
        p.off += o;
        B.patches.push_back(p);
      }
      for (CfiEntry e : A.cfi) {
        e.dst += o;
        if (e.src >= 0) e.src += o;
        else e.src = -1 - (-1 - e.src + c * nside);
        e.cpatch += c * npc;
        e.fpatch += c * np;
        B.cfi.push_back(e);
      }
      for (long long key : A.cfi_key) B.cfi_key.push_back(key + c * key_span);
      for (long long v : A.cfi_side) B.cfi_side.push_back(v + o);
      for (CopyEntry e : A.copy) {
        e.dst += o;
        e.src += o;
        B.copy.push_back(e);
      }
      for (RefluxEntry e : A.reflux) {
        e.coff += o;
        e.cpatch += c * np;
        for (int f = 0; f < 6; ++f)
          if (e.fpatch[f] >= 0) e.fpatch[f] += c * npf;
        B.reflux.push_back(e);
      }
      for (XferBlock x : A.xfer) {
        x.fpatch += c * npf;
        x.cpatch += c * np;
        B.xfer.push_back(x);
      }
    }
    B.dev.xfer_max[0] = A.dev.xfer_max[0];
    B.dev.xfer_max[1] = A.dev.xfer_max[1];
    B.dev.xfer_max[2] = A.dev.xfer_max[2];
  }
  s->mg = h->mg;
  for (size_t m = 0; m < s->mg.size(); ++m) {
    MgGrid& g = s->mg[m];
    g.d_patch = nullptr;
    if (m == 0) {
      g.cstride = stride;
      g.nelems = stride * k;
    } else {
      g.cstride = (h->mg[m].nelems + 63) / 64 * 64;
      g.nelems = g.cstride * k;
    }
  }
  // valid flags in the order the patches are laid out: level by level, within a level the
  // replicas one after another
  {
    size_t q = 0;
    for (int l = 0; l < h->L; ++l) {
      size_t cells = 0;
      for (const PatchDesc& p : h->lev[l].patches) cells += (size_t)p.n[0] * p.n[1] * p.n[2];
      for (int c = 0; c < k; ++c)
        s->im_valid.insert(s->im_valid.end(), h->im_valid.begin() + q, h->im_valid.begin() + q + cells);
      q += cells;
    }
  }
  const amr_status st = upload_hierarchy(s.get(), err);
  if (st != AMR_OK) {
    free_hierarchy(s.get());
    return st;
  }
  *out = s.release();
  return AMR_OK;
}

// Device copies of the work lists and masks, made on the first call that needs the GPU
// (hierarchy creation and the index maps work without one).
// Data migration plan (Sec. 5.4, last paragraph): the cells of new level l inside a box of
// old level l are copied (one block per intersecting pair of boxes); every other cell gets
// the AMRCFI value from new level l-1 (filled before level l), with the window of Sec. 5.2
// (centred on the parent, slid inward at the physical boundary).  Level 0 is one block.
amr_status migrate_plan(const amr_hierarchy* oh, const amr_hierarchy* nh, std::vector<MigrateLevel>& plan,
                        std::string& err) {
  const int D = nh->D, r = nh->r;
  if (oh->D != D || oh->r != r || oh->ncomp != 1 || nh->ncomp != 1) {
    err = "migration: the hierarchies need the same dimension and ratio (and no stacking)";
    return AMR_ERR_INVALID_ARG;
  }
  for (int e = 0; e < D; ++e)
    if (oh->n0[e] != nh->n0[e]) {
      err = "migration: the hierarchies need the same level-0 domain";
      return AMR_ERR_INVALID_ARG;
    }
  plan.assign(nh->L, {});
  for (int l = 0; l < nh->L; ++l) {
    const LevelHost& N = nh->lev[l];
    MigrateLevel& M = plan[l];
    const bool has_old = l < oh->L;
    LevelMap omap;
    if (has_old) omap.build(oh->lev[l].boxes, D);
    for (size_t k = 0; k < N.boxes.size(); ++k) {
      const Box& nb = N.boxes[k];
      if (has_old)
        for (size_t q = 0; q < oh->lev[l].boxes.size(); ++q) {
          const Box& ob = oh->lev[l].boxes[q];
          MigrateBlock blk{};
          blk.npatch = (int)k;
          blk.opatch = (int)q;
          bool ok = true;
          for (int e = 0; e < 3; ++e) { blk.lo[e] = 0; blk.hi[e] = 0; }
          for (int e = 0; e < D; ++e) {
            blk.lo[e] = std::max(nb.lo[e], ob.lo[e]);
            blk.hi[e] = std::min(nb.hi[e], ob.hi[e]);
            ok = ok && blk.lo[e] <= blk.hi[e];
          }
          if (ok) M.blocks.push_back(blk);
        }
      if (l == 0) continue;  // level 0 is the domain in both hierarchies
      const LevelHost& C = nh->lev[l - 1];
      LevelMap cmap;
      cmap.build(C.boxes, D);
      const PatchDesc& p = N.patches[k];
      int g[3] = {0, 0, 0};
      for (g[2] = (D == 3 ? nb.lo[2] : 0); g[2] <= (D == 3 ? nb.hi[2] : 0); ++g[2])
        for (g[1] = nb.lo[1]; g[1] <= nb.hi[1]; ++g[1])
          for (g[0] = nb.lo[0]; g[0] <= nb.hi[0]; ++g[0]) {
            if (has_old && omap.at(g) >= 0) continue;
            CfiEntry ce{};
            ce.dst = cell_off(p, D, g[0] - p.lo[0], g[1] - p.lo[1], D == 3 ? g[2] - p.lo[2] : 0);
            ce.fpatch = (int)k;
            int start[3] = {0, 0, 0};
            for (int e = 0; e < 3; ++e) { ce.pos[e] = 0; ce.sub[e] = 0; }
            for (int e = 0; e < D; ++e) {
              const int par = g[e] / r;  // cells of a box are inside the domain: g >= 0
              const int s0 = std::min(std::max(par - 2, 0), C.ndom[e] - CFI_W);
              start[e] = s0;
              ce.pos[e] = (signed char)(par - s0);
              ce.sub[e] = (signed char)(g[e] - r * par);
            }
            const int cp0 = cmap.at(start);
            bool single = cp0 >= 0;
            if (single) {
              const PatchDesc& cpd = C.patches[cp0];
              for (int e = 0; e < D; ++e)
                single = single && start[e] >= cpd.lo[e] && start[e] + CFI_W - 1 <= cpd.lo[e] + cpd.n[e] - 1;
            }
            if (single) {
              const PatchDesc& cpd = C.patches[cp0];
              ce.cpatch = cp0;
              ce.src = cell_off(cpd, D, start[0] - cpd.lo[0], start[1] - cpd.lo[1], D == 3 ? start[2] - cpd.lo[2] : 0);
            } else {
              ce.cpatch = -1;
              ce.src = -1 - (long long)(M.side.size() / (D == 3 ? 125 : 25));
              for (int wz = 0; wz < (D == 3 ? CFI_W : 1); ++wz)
                for (int wy = 0; wy < CFI_W; ++wy)
                  for (int wx = 0; wx < CFI_W; ++wx) {
                    int c[3] = {start[0] + wx, start[1] + wy, D == 3 ? start[2] + wz : 0};
                    const int q2 = cmap.at(c);
                    if (q2 < 0) {
                      err = "migration: an AMRCFI window of new level " + std::to_string(l) + " leaves new level " +
                            std::to_string(l - 1) + " (the new hierarchy is not properly nested)";
                      return AMR_ERR_NESTING;
                    }
                    const PatchDesc& cpd = C.patches[q2];
                    M.side.push_back(cell_off(cpd, D, c[0] - cpd.lo[0], c[1] - cpd.lo[1], D == 3 ? c[2] - cpd.lo[2] : 0));
                  }
            }
            M.cfi.push_back(ce);
            for (int e = 0; e < D; ++e) {
              M.cells.push_back(g[e]);
              M.starts.push_back(start[e]);
            }
          }
    }
  }
  return AMR_OK;
}

amr_status upload_hierarchy(amr_hierarchy* h, std::string& err) {
  if (h->on_device) return AMR_OK;
  std::vector<unsigned char> valid(h->nelems, 0);
  {
    size_t q = 0;
    for (int l = 0; l < h->L; ++l)
      for (const PatchDesc& p : h->lev[l].patches)
        for (int z = 0; z < p.n[2]; ++z)
          for (int y = 0; y < p.n[1]; ++y)
            for (int x = 0; x < p.n[0]; ++x) valid[cell_off(p, h->D, x, y, z)] = (unsigned char)h->im_valid[q++];
  }
  try {
    for (int l = 0; l < h->L; ++l) {
      LevelHost& L = h->lev[l];
      L.d_patches = upload(L.patches);
      L.dev.cfi = upload(L.cfi);
      L.dev.ncfi = (long long)L.cfi.size();
      {
        const std::vector<CfiGroup> g = cfi_groups(L.cfi, L.cfi_key, h->r, h->D);
        L.dev.cfig = upload(g);
        L.dev.ncfig = (long long)g.size();
      }
      L.dev.cfi_side = upload(L.cfi_side);
      L.dev.copy = upload(L.copy);
      L.dev.ncopy = (long long)L.copy.size();
      L.dev.cicf = upload(L.cicf);
      L.dev.ncicf = (int)L.cicf.size();
      L.dev.cic_cstart = upload(L.cic_cstart);
      L.dev.ncic_comp = L.cic_cstart.empty() ? 0 : (int)L.cic_cstart.size() - 1;
      L.dev.cic_slot = upload(L.cic_slot);
      L.dev.cic_chunks = upload(L.cic_chunks);
      L.dev.cic_ccstart = upload(L.cic_ccstart);
      L.dev.ncic_chunks = (int)L.cic_chunks.size();
      if (!L.cic_chunks.empty() &&
          cudaMalloc(&L.dev.cic_psum, sizeof(double) * L.cic_chunks.size()) != cudaSuccess)
        throw std::runtime_error("cudaMalloc failed");
      L.dev.reflux = upload(L.reflux);
      L.dev.nreflux = (long long)L.reflux.size();
      L.dev.xfer = upload(L.xfer);
      L.dev.nxfer = (int)L.xfer.size();
    }
    for (auto& g : h->mg) {
      std::vector<PatchDesc> reps(h->ncomp, g.patch);
      for (int c = 0; c < h->ncomp; ++c) reps[c].off = g.patch.off + c * g.cstride;
      g.d_patch = upload(reps);
    }
    h->d_valid = upload(valid);
    {
      std::vector<unsigned long long> z(2 * (size_t)h->ncomp, 0ull);
      h->d_fxs = upload(z);
      h->d_cnorm = upload(z);
    }
    if (cudaMalloc(&h->d_red, sizeof(double) * 2 * 8192) != cudaSuccess) throw std::runtime_error("cudaMalloc failed");
    if (cudaMalloc(&h->d_scalar, sizeof(double) * 16) != cudaSuccess) throw std::runtime_error("cudaMalloc failed");
    if (cudaMallocHost(&h->h_scalar, sizeof(double) * 16) != cudaSuccess) throw std::runtime_error("cudaMallocHost failed");
  } catch (const std::exception& ex) {
    cudaGetLastError();
    err = ex.what();
    return AMR_ERR_OOM;
  }
  h->on_device = true;
  return AMR_OK;
}

void free_hierarchy(amr_hierarchy* h) {
  if (!h->on_device) return;
  for (auto& L : h->lev) {
    cudaFree(L.d_patches);
    cudaFree(L.dev.cfi);
    cudaFree(L.dev.cfig);
    cudaFree(L.dev.cfi_side);
    cudaFree(L.dev.copy);
    cudaFree(L.dev.cicf);
    cudaFree(L.dev.cic_cstart);
    cudaFree(L.dev.cic_chunks);
    cudaFree(L.dev.cic_ccstart);
    cudaFree(L.dev.cic_psum);
    cudaFree(L.dev.cic_band);
    cudaFree(L.dev.cic_slot);
    cudaFree(L.dev.cic_y);
    cudaFree(L.dev.reflux);
    cudaFree(L.dev.xfer);
  }
  for (auto& g : h->mg) cudaFree(g.d_patch);
  cudaFree(h->d_valid);
  cudaFree(h->d_fxs);
  cudaFree(h->d_cnorm);
  cudaFree(h->d_red);
  cudaFree(h->d_scalar);
  cudaFree(h->d_tz);
  if (h->h_scalar) cudaFreeHost(h->h_scalar);
}

// Eqs. (velBCHomoDiri5th), (Neumann5): coefficient of interior cell m in ghost layer 1 / 2
static const double GC[2][2][4] = {{{-77.0 / 12.0, 43.0 / 12.0, -17.0 / 12.0, 3.0 / 12.0},
                                    {-505.0 / 12.0, 335.0 / 12.0, -145.0 / 12.0, 27.0 / 12.0}},
                                   {{5.0 / 10.0, 9.0 / 10.0, -5.0 / 10.0, 1.0 / 10.0},
                                    {-75.0 / 10.0, 145.0 / 10.0, -75.0 / 10.0, 15.0 / 10.0}}};

void finish_view(LevelView& v) {
  v.hd = v.h;
  v.hf = (float)v.h;
  v.inv12h2 = 1.0 / (12.0 * v.h * v.h);
  v.inv12h = 1.0 / (12.0 * v.h);
  v.inv12h2_f = (float)v.inv12h2;
  v.inv12h_f = (float)v.inv12h;
  v.invh = 1.0 / v.h;
  v.invh_f = (float)v.invh;
  for (int f = 0; f < 6; ++f) {
    const int t = v.bc[f] == 1 ? 1 : 0;
    // the cell owning the face reads ghost 1 with weight 16 and ghost 2 with weight -1; the
    // next cell reads ghost 1 with weight -1 (Eq. discreteOps c)
    v.dcorr[f][0] = 16.0 * GC[t][0][0] - GC[t][1][0];
    v.dcorr[f][1] = -GC[t][0][1];
    v.dcorr_f[f][0] = (float)v.dcorr[f][0];
    v.dcorr_f[f][1] = (float)v.dcorr[f][1];
  }
}

LevelView level_view(const amr_hierarchy* h, int l, const int* bc_types) {
  LevelView v{};
  const LevelHost& L = h->lev[l];
  v.patches = L.d_patches;
  v.npatch = (int)L.patches.size();
  v.D = h->D;
  v.h = L.h;
  for (int e = 0; e < 3; ++e) { v.ndom[e] = L.ndom[e]; v.maxn[e] = L.maxn[e]; }
  v.ncells = 0.0;
  for (const PatchDesc& p : L.patches) v.ncells += (double)p.n[0] * p.n[1] * p.n[2];
  for (int f = 0; f < 6; ++f) {
    v.bc[f] = (f < 2 * h->D && bc_types) ? bc_types[f] : 0;
    v.bc_off[f] = (f < 2 * h->D) ? h->bc_off[(size_t)l * 2 * h->D + f] : 0;
    // leading transverse extent of face f's array
    int d = f / 2, lead = -1;
    for (int e = 0; e < h->D; ++e)
      if (e != d) { lead = e; break; }
    v.bc_pitch[f] = (f < 2 * h->D && lead >= 0) ? L.ndom[lead] : 1;
  }
  v.fxs = h->ncomp > 1 ? h->d_fxs : (h->d_scalar ? reinterpret_cast<unsigned long long*>(h->d_scalar + 8) : nullptr);
  v.p0 = L.patches.front();
  v.ncomp = h->ncomp;
  v.cstride = h->cstride;
  v.active = h->ncomp > 1 ? h->d_active : nullptr;
  finish_view(v);
  return v;
}

}  // namespace amr4
