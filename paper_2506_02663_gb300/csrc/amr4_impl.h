// Internal data structures of libamr4 (host C++ and CUDA).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/amr4.h"

namespace amr4 {

constexpr int NG = 2;         // ghost layers (Sec. 3, paragraph after Eq. appProj)
constexpr int CFI_W = 5;      // AMRCFI window width (degree-4 reconstruction)
constexpr int MIN_BOX = 4;    // one-sided ghost formulas read 4 interior cells
constexpr int NEST_MARGIN = 3;
constexpr int MAX_BOTTOM = 1024;

// One padded patch of a composite field (device-visible, trivially copyable).
struct PatchDesc {
  long long off;   // element offset of the padded patch
  long long sy;    // y stride (elements)
  long long sz;    // z stride (elements; = sy*(ny+4) in 3-D, 0 in 2-D)
  int n[3];        // interior extents (1 in unused dimensions)
  int lo[3];       // global index of interior cell (0,0,0) at its level
};

// Level description passed by value to kernels.
struct LevelView {
  const PatchDesc* patches;  // device array
  int npatch;
  int D;
  int ndom[3];
  int maxn[3];               // largest interior extents (launch shape)
  double h;
  int bc[6];                 // boundary type per face
  long long bc_off[6];       // offsets of this level's faces inside a bc array
  long long bc_pitch[6];     // leading extent of each face array (transverse dim 0)
  double ncells;             // interior cells over all patches (host bookkeeping)
  // per-level constants precomputed on the host, in both precisions, so that FP32 kernels
  // execute no FP64 instruction per cell
  double hd, inv12h2, inv12h, invh;
  float hf, inv12h2_f, inv12h_f, invh_f;
  double dcorr[6][2];        // Jacobi diagonal correction (x 12 h^2) at distance 0 / 1 from face f
  float dcorr_f[6][2];
  // device scratch of the fixed-point FP64 residual (two words: largest |x| as IEEE bits,
  // out-of-frame flag); null for views that are not a hierarchy level
  unsigned long long* fxs;
  // host-side copy of the first patch (the only one of a single-patch level): kernels fed by
  // tensor-map copies need its offset and strides on the host
  PatchDesc p0;
  // stacked component batches: the level holds ncomp replicas of its patches, replica c at
  // element offset c * cstride (ncomp = 1, cstride = 0 otherwise); fxs then holds two
  // words per component
  int ncomp;
  long long cstride;
  const int* active;  // stacked batches: replicas still iterating (nullptr: all)
};

void finish_view(LevelView& v);  // fills the precomputed constants from h and bc

// AMRCFI ghost cell: dst = fine field offset; src >= 0: field offset of the window's first
// coarse cell in coarse patch cpatch; src < 0: -(1+k) with the 5^D offsets at side[k*5^D].
struct CfiEntry {
  long long dst;
  long long src;
  int cpatch;
  signed char pos[3];
  signed char sub[3];
  signed char dir;    // dimension along which the ghost lies outside its fine patch
  signed char layer;  // -L: L cells below the patch's low side, +L: above its high side
  int fpatch;         // fine patch (index within its level)
};

// The 2^D fine CF ghost cells of one coarse parent (ratio 2, one face of one fine patch): they
// share the parent's 5^D window, so the interpolation runs once per parent, dimension by
// dimension.  Child c = sub_x + 2 sub_y + 4 sub_z; dst < 0 where a child is absent.
struct CfiGroup {
  long long src;     // window origin in its coarse patch, or -1 - index of its side table
  long long dst[8];  // fine ghost cells
  int cpatch;
  signed char pos[3];
  signed char pad;
};

// One coarse-fine interface face of a level (Sec. 6.4, Eq. correctingFaceAvg): the CF ghost
// of the first layer across it, step = side x the patch stride along the face normal (the
// interior cell next to the face is ghost - step, the second ghost layer ghost + step), the
// normal dimension and the side (+1: the interior cell's high face).
struct CicFace {
  long long ghost;
  long long step;
  int dir;
  int side;
};

// A chunk of one component's interface faces [begin, end), one block of the face passes.
struct CicChunk {
  int comp;
  int begin;
  int end;
  int pad;
};

struct CopyEntry {
  long long dst;
  long long src;
};

// Coarse valid cell with >= 1 coarse-fine face (COH-3).
struct RefluxEntry {
  long long coff;   // coarse field offset of the cell
  int cpatch;       // coarse patch
  int faces;        // bit 2d+side
  int g[3];         // coarse global index
  int fpatch[6];    // fine patch that covers the neighbour across face 2d+side
};

// Fine box x coarse box intersection, used for restriction / average-down / prolongation.
struct XferBlock {
  int fpatch;
  int cpatch;
  int clo[3];  // coarse global region [clo, chi]
  int chi[3];
};

struct Box {
  int lo[3];
  int hi[3];
};

struct DeviceLists {
  CfiEntry* cfi = nullptr;
  long long* cfi_side = nullptr;
  long long ncfi = 0;
  CfiGroup* cfig = nullptr;  // the same ghosts grouped by coarse parent (ratio 2)
  long long ncfig = 0;
  CopyEntry* copy = nullptr;
  long long ncopy = 0;
  CicFace* cicf = nullptr;  // coarse-fine interface faces, grouped by connected component
  int* cic_cstart = nullptr;
  int ncicf = 0;
  int ncic_comp = 0;
  CicChunk* cic_chunks = nullptr;  // at least one chunk per component
  int* cic_ccstart = nullptr;      // chunks of component c: [ccstart[c], ccstart[c+1])
  double* cic_psum = nullptr;      // one partial sum per chunk
  int ncic_chunks = 0;
  // 3-D interface ghosts: the distinct coarse cells of the level's AMRCFI windows (field
  // offsets, ascending) and scratch for their two time combinations, indexed by offset -
  // cic_base over the coarse level's span; made by the first amr_cic_ghosts call
  long long* cic_band = nullptr;
  long long ncic_band = 0;
  long long cic_base = 0;
  double* cic_y = nullptr;  // 2 x cic_span doubles
  long long cic_span = 0;
  long long* cic_slot = nullptr;  // per face, see LevelHost::cic_slot
  RefluxEntry* reflux = nullptr;
  long long nreflux = 0;
  XferBlock* xfer = nullptr;  // blocks between this level (coarse) and level+1
  int nxfer = 0;
  int xfer_max[3] = {1, 1, 1};  // largest coarse region extent
};

struct LevelHost {
  std::vector<Box> boxes;
  int ndom[3] = {1, 1, 1};
  double h = 0.0;
  std::vector<PatchDesc> patches;
  int first_patch = 0;  // global patch index of the first patch
  PatchDesc* d_patches = nullptr;
  std::vector<CfiEntry> cfi;
  std::vector<long long> cfi_side;
  std::vector<long long> cfi_key;  // per CF ghost: its coarse parent and face (grouping key)
  std::vector<CopyEntry> copy;
  // coarse-fine interface faces (one per first-layer CF ghost), grouped by the connected
  // component of their patch (components in ascending order of their smallest box index);
  // faces of component c are [cic_cstart[c], cic_cstart[c+1]); cic_cell holds D global
  // indices per face (the interior cell), cic_comp the component of each face
  std::vector<CicFace> cicf;
  std::vector<int> cic_cstart;
  std::vector<int> cic_cell;
  std::vector<int> cic_comp;
  std::vector<CicChunk> cic_chunks;
  std::vector<int> cic_ccstart;
  // components that are a single box: that box's index (-1 for a component of several
  // boxes), and per face its slot in the boundary-data layout of the one-level problem whose
  // domain is the box (-1 for faces of multi-box components)
  std::vector<int> cic_comp_box;
  std::vector<long long> cic_slot;
  std::vector<RefluxEntry> reflux;  // this level's coarse cells bordering level+1
  std::vector<XferBlock> xfer;      // this level (coarse) <-> level+1 (fine)
  DeviceLists dev;
  int maxn[3] = {1, 1, 1};
};

// A single-box grid of the level-0 multigrid pyramid.
struct MgGrid {
  int n[3] = {1, 1, 1};
  double h = 0.0;
  PatchDesc patch{};
  PatchDesc* d_patch = nullptr;  // ncomp replicas of patch, replica c at offset c * cstride
  long long nelems = 0;          // elements of the grid's arrays (all replicas)
  long long cstride = 0;         // element stride between replicas
};

}  // namespace amr4

struct amr_hierarchy {
  int D = 2;
  int r = 2;
  int n0[3] = {1, 1, 1};
  double h0 = 0.0;
  int L = 0;  // number of levels
  std::vector<amr4::LevelHost> lev;
  long long nelems = 0;
  int npatch = 0;
  std::vector<amr_patch_info> pinfo;
  unsigned char* d_valid = nullptr;  // composite layout: 1 on valid interior cells
  std::vector<long long> bc_off;     // nlevels*2D + 1
  std::vector<amr4::MgGrid> mg;      // level-0 multigrid grids (mg[0] = level 0 itself)
  // index maps (host)
  std::vector<int> im_valid, im_component, im_code, im_src, im_aux;
  std::vector<long long> im_cfi_cell;
  std::vector<int> im_cfi_start, im_cfi_pos, im_cfi_sub;
  std::vector<int> im_reflux_cell, im_reflux_faces;
  // CFI weights W[pos][sub][a] (exact rationals rounded once), ratio r
  std::vector<double> cfi_w;
  // reduction scratch (device)
  double* d_red = nullptr;       // partials
  double* d_scalar = nullptr;    // a few device scalars
  double* h_scalar = nullptr;    // pinned host mirror
  double* d_tz = nullptr;        // G/D transposes: 3 composite fields (allocated on first use)
  bool cfi_const_ready = false;  // AMRCFI weights copied to the device constant banks
  bool on_device = false;
  // stacked component batch (built by stack_hierarchy): every patch and work list replicated
  // ncomp times, replica c of the composite layout at element offset c * cstride
  int ncomp = 1;
  long long cstride = 0;            // elements of one replica (nelems / ncomp)
  unsigned long long* d_fxs = nullptr;   // fixed-point residual words, two per component
  unsigned long long* d_cnorm = nullptr; // per-component residual and right-hand-side norms (IEEE bits)
  const int* d_active = nullptr;         // stacked batches: replicas still iterating (set by the solve)
};

namespace amr4 {
// hierarchy.cpp
amr_status build_hierarchy(const amr_hierarchy_desc* desc, amr_hierarchy* h, std::string& err);
void free_hierarchy(amr_hierarchy* h);
amr_status upload_hierarchy(amr_hierarchy* h, std::string& err);
// A new hierarchy holding k replicas of h (same geometry): patches, work lists and masks
// repeated with element offsets c * stride (stride = h's composite length rounded up to 64
// elements), patch indices shifted per replica; uploaded to the device.
amr_status stack_hierarchy(const amr_hierarchy* h, int k, amr_hierarchy** out, std::string& err);
// Data migration after regridding: per level of the new hierarchy, the blocks copied from the
// old hierarchy's same level (intersections of a new and an old box, level index space) and
// the AMRCFI entries of the other new cells (windows in the new level l-1; side tables for
// windows over several patches).
struct MigrateBlock {
  int npatch;  // patch of the new level
  int opatch;  // patch of the old level
  int lo[3];
  int hi[3];
};
struct MigrateLevel {
  std::vector<MigrateBlock> blocks;
  std::vector<CfiEntry> cfi;
  std::vector<long long> side;
  std::vector<int> cells;   // dim ints per AMRCFI entry: the new cell (global index)
  std::vector<int> starts;  // dim ints per AMRCFI entry: the window's first coarse cell
};
amr_status migrate_plan(const amr_hierarchy* oh, const amr_hierarchy* nh, std::vector<MigrateLevel>& plan,
                        std::string& err);
void set_error(const std::string& msg);
const char* get_error();
void cfi_weights_exact(int r, std::vector<double>& w);  // [pos][sub][a], 5 x r x 5
LevelView level_view(const amr_hierarchy* h, int l, const int* bc_types);
}  // namespace amr4
