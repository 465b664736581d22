// sweep3d.cuh -- 3-D level operator on single-patch levels, fed by tensor-map TMA copies.
//
// The weighted-Jacobi sweep of Sec. 6.5 (true diagonal, omega), the residual f - A x and the
// operator A x = alpha x + beta L x of Eq. (discreteOps) on a single-patch 3-D level whose
// x extent is a multiple of 64 cells and whose y extent is a multiple of the tile height TY.
//
// Design (GB300): a block owns a 64 x TY tile column and marches up z through one chunk of
// planes.  Three warp roles share a ring of S shared-memory slots, one plane per slot:
//   * producer (one thread): streams the planes of x (the tile plus its two-cell halo, a
//     68 x (TY + 4) box of the padded patch) into the ring with tensor-map TMA copies
//     (cp.async.bulk.tensor), one per plane, completing on the slot's "full" mbarrier (the
//     first sweep from x = 0, which reads f alone, streams f the same way);
//   * fixer (one warp, only in blocks that touch a domain face): writes the physical ghost
//     values (Eqs. velBCHomoDiri5th, Neumann5, homogeneous data -- never stored in global
//     memory) into the slot's halo columns, halo rows and, at a z face, the ghost planes,
//     from the staged cells next to the face, then signals the slot's "ready" mbarrier;
//   * consumers (TY / RW warps; warp w owns RW tile rows, lane l the cells 2l, 2l+1 of a
//     row): read every neighbour of the 13-point stencil from the ring (planes k-2 .. k+2),
//     with one 8- or 16-byte shared load per neighbour pair, and store one pair per row; f
//     is read from global memory two planes ahead into registers, which keeps the slots
//     small enough for three blocks per SM.  A slot is released through its "empty"
//     mbarrier once plane k+2 no longer needs it.
// The consumer loop has no face branch and no block-wide barrier; up to S - 5 planes are in
// flight per block.  Stored ghost values (coarse-fine, copies) arrive with the halo.  The
// Jacobi factor comes from the 125-entry distance-class table.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets bit 0 of g_sweep3d_err,
// and the warp stops (the producer first waits, again bounded, for the copies it issued).
//
// The stencil sums are formed in the same order and with the same multiply-adds as
// k_level_op3d_zc; the ghost values are the same formulas.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace amr4 {
namespace sw3 {

constexpr int TX = 64;        // tile width (cells); lane l owns cells 2l, 2l+1
constexpr int XW = TX + 4;    // slot row: padded columns i0 .. i0 + 67 (cells i0-2 .. i0+65)
constexpr int WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// try_wait with a suspend-time hint: the warp sleeps until the phase completes or about
// 0.5 us pass, instead of spinning on the issue slots other warps need
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 500;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the completion of the phase with the given parity: gives up after about
// one second (or WAIT_LIMIT polls, whichever comes first)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 1; it < WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}
// 4-D tiled TMA load of the box at (c0, c1, c2, c3) of the tensor map into shared memory
// (128-byte aligned), completing its bytes on the mbarrier; dimension 3 is the replica of a
// stacked component batch (extent 1 otherwise)
__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(tm)) : "memory");
}

template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
};
template <>
struct Pair<double> {
  using V = double2;
};

template <typename T>
__device__ __forceinline__ typename Pair<T>::V ld2(const T* s) {
  return *reinterpret_cast<const typename Pair<T>::V*>(s);
}
template <typename T>
__device__ __forceinline__ void st2(T* g, typename Pair<T>::V v) {
  *reinterpret_cast<typename Pair<T>::V*>(g) = v;
}

// ghost value of layer ``layer`` (0 = next to the face) from the four cells a0 (next to the
// face) .. a3 inward
template <typename T>
__device__ __forceinline__ T ghost4(int type, int layer, T a0, T a1, T a2, T a3) {
  T v = T(0);
  v += gcoef<T>(type, layer, 0) * a0;
  v += gcoef<T>(type, layer, 1) * a1;
  v += gcoef<T>(type, layer, 2) * a2;
  v += gcoef<T>(type, layer, 3) * a3;
  return v;
}

// elements of a region of ``rows`` slot rows, rounded up to 128 bytes (TMA destinations)
template <typename T>
__host__ __device__ constexpr int region_elems(int rows) {
  return (int)(((size_t)rows * XW * sizeof(T) + 127) / 128 * 128 / sizeof(T));
}
template <int TY, typename T>
__host__ __device__ constexpr size_t slot_elems(bool needx, bool needf) {
  return (needx ? (size_t)region_elems<T>(TY + 4) : 0) + (needf ? (size_t)region_elems<T>(TY) : 0);
}

template <typename T, int MODE, int TY, int S>
constexpr size_t smem_bytes() {
  return (size_t)S * slot_elems<TY, T>(MODE != OP_JACOBI0, MODE == OP_JACOBI0) * sizeof(T) + 3 * S * sizeof(unsigned long long) +
         128 * sizeof(T);
}

}  // namespace sw3

// Set (bit 0) when a bounded mbarrier wait of k_sweep3d ran out; read and cleared by the host.
__device__ unsigned g_sweep3d_err = 0u;

namespace sw3 {
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
}  // namespace sw3

// Residual restriction (multigrid down leg): the residual f - A x of each fine cell, summed
// over the 2 x 2 x 2 children of every coarse cell in the order and with the arithmetic of
// cell_restrict, times 1/8, into the coarse grid's right-hand side.
constexpr int OP_RESTRICT = 4;

// MODE: OP_JACOBI0 (x = 0: out = w f), OP_JACOBI, OP_RESID (vmask: valid cells only),
// OP_APPLY, OP_RESTRICT (outc: the coarse grid, layout cpd, replica stride ccs; even chunk
// boundaries; RW = 2, so that a warp's two rows are one coarse row).  tmx / tmf: tensor maps of x and f over the padded patch (dimensions: pitch,
// n_y + 4, n_z + 4; boxes 68 x (TY + 4) x 1 and 68 x TY x 1).  Grid: ntiles tile columns x
// nch z chunks (chunk c: planes [c nz / nch, (c + 1) nz / nch), at least four planes each:
// nch <= nz / 4); block 32 (TY / RW + 2).
template <typename T, int MODE, int TY, int RW, int S>
__global__ void __launch_bounds__(32 * (TY / RW + 2), sizeof(T) == 4 ? 3 : 2)  // FP32: three blocks per SM
    k_sweep3d(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmf, LevelView lv, int ntx,
              int ntiles, int nch, const T* __restrict__ f, T* __restrict__ out, T alpha, T beta, T omega,
              const unsigned char* __restrict__ vmask, const unsigned* __restrict__ gate, T* __restrict__ outc,
              PatchDesc cpd, long long ccs) {
  using namespace sw3;
  using V = typename Pair<T>::V;
  unsigned* err = &g_sweep3d_err;
  constexpr bool NEEDX = MODE != OP_JACOBI0;
  constexpr bool NEEDF = MODE != OP_APPLY;
  constexpr bool FTMA = MODE == OP_JACOBI0;  // f through the ring (else prefetched into registers)
  constexpr int NCW = TY / RW;               // consumer warps
  constexpr int XH = TY + 4;                 // slot rows of x
  constexpr int XSZ = NEEDX ? region_elems<T>(XH) : 0;
  constexpr int SLOT = XSZ + (FTMA ? region_elems<T>(TY) : 0);
  static_assert(TY % RW == 0 && S >= 8, "tile rows must split into warps; the ring needs eight slots");
  static_assert(MODE != OP_RESTRICT || RW == 2, "restriction: a warp's two rows form one coarse row");
  extern __shared__ __align__(128) unsigned char sw3_smem[];
  T* ring = reinterpret_cast<T*>(sw3_smem);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(sw3_smem + (size_t)S * SLOT * sizeof(T));
  unsigned long long* ready = full + S;
  unsigned long long* empty = ready + S;
  T* wt = reinterpret_cast<T*>(empty + S);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T inv = pick<T>(lv.inv12h2, lv.inv12h2_f);
  if (MODE == OP_JACOBI || MODE == OP_JACOBI0) {
    for (int q = tid; q < 125; q += blockDim.x) {
      const int cls[3] = {q % 5, (q / 5) % 5, q / 25};
      T acc = T(-90);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (cls[d]) acc += pick<T>(lv.dcorr[2 * d + (cls[d] - 1) / 2][(cls[d] - 1) % 2],
                                   lv.dcorr_f[2 * d + (cls[d] - 1) / 2][(cls[d] - 1) % 2]);
      wt[q] = omega / (alpha + beta * inv * acc);
    }
  }
  // stacked component batches: the grid holds ncomp equal parts, part c on replica c (tensor
  // coordinate 3 = c; its patch offset for the stores and f)
  const int bpc = gridDim.x / lv.ncomp, comp = blockIdx.x / bpc, blk = blockIdx.x % bpc;
  PatchDesc p = lv.p0;
  p.off += comp * lv.cstride;
  const int nz = p.n[2];
  const int tile = blk % ntiles, chunk = blk / ntiles;
  const int ev = MODE == OP_RESTRICT ? ~1 : ~0;  // restriction: chunks of whole plane pairs
  const int ka = (int)(((long long)chunk * nz) / nch) & ev, kb = (int)(((long long)(chunk + 1) * nz) / nch) & ev;
  const int i0 = (tile % ntx) * TX, j0 = (tile / ntx) * TY;
  const int lz = p.lo[2], nzd = lv.ndom[2];
  const int gx0 = p.lo[0] + i0, gy0 = p.lo[1] + j0;
  const bool fxl = gx0 == 0, fxh = gx0 + TX == lv.ndom[0], fyl = gy0 == 0, fyh = gy0 + TY == lv.ndom[1];
  const bool fzl = lz + ka == 0, fzh = lz + kb == nzd;
  const bool fix = NEEDX && (fxl || fxh || fyl || fyh || fzl || fzh);  // block-uniform
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&ready[q], 1);
      mbar_init(&empty[q], NCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (ka >= kb) return;
  pdl_wait();
  // converged replica of a stacked batch (the flags are written by the stopping test of the
  // previous graph phase: read after the wait)
  if (lv.active != nullptr && !lv.active[comp]) return;
  const int kfirst = NEEDX ? ka - 2 : ka;
  const int np = NEEDX ? (kb - ka) + 4 : (kb - ka);  // planes through the ring
  if (gate != nullptr && gate[4 * comp] == 0u) return;  // gated launch: runs only when the flag is set

  if (warp == NCW) {
    // ---------------------------------------------------------------- producer (one thread)
    if (lane != 0) return;
    if (NEEDX) tma_prefetch_desc(&tmx);
    if (FTMA) tma_prefetch_desc(&tmf);
    int q = 0;
    bool ok = true;
    for (; q < np; ++q) {
      const int sl = q % S, use = q / S, k = kfirst + q;
      if (use > 0 && !mbar_wait(&empty[sl], (unsigned)((use - 1) & 1))) {
        ok = false;
        break;
      }
      const bool ghost = NEEDX && (lz + k < 0 || lz + k >= nzd);  // z ghost plane: the fixer writes it
      const bool wf = FTMA && k >= ka && k < kb;
      if (ghost) {
        mbar_arrive(&full[sl]);
        continue;
      }
      mbar_expect_tx(&full[sl], (unsigned)((NEEDX ? XH * XW : 0) + (wf ? TY * XW : 0)) * (unsigned)sizeof(T));
      T* sx = ring + (size_t)sl * SLOT;
      // padded coordinates: column i0 (cell i0 - 2), row j0 (cell j0 - 2) / j0 + 2, plane k + 2
      if (NEEDX) tma_load4(sx, &tmx, i0, j0, k + NG, comp, &full[sl]);
      if (wf) tma_load4(sx + XSZ, &tmf, i0, j0 + NG, k + NG, comp, &full[sl]);
    }
    if (!ok) atomicOr(err, 1u);
    // the block must not end while copies into its shared memory are in flight: wait
    // (bounded) for the last copies issued into every slot (none is reused after them)
    for (int t = max(0, q - S); t < q; ++t) mbar_wait(&full[t % S], (unsigned)((t / S) & 1));
    return;
  }

  if (warp == NCW + 1) {
    // ---------------------------------------------------------------- fixer (one warp)
    if (!fix) return;
    const int txl = lv.bc[0], txh = lv.bc[1], tyl = lv.bc[2], tyh = lv.bc[3], tzl = lv.bc[4], tzh = lv.bc[5];
    auto slot = [&](int q) -> T* { return ring + (size_t)(q % S) * SLOT; };
    auto wait_full = [&](int q) -> bool { return mbar_wait(&full[q % S], (unsigned)((q / S) & 1)); };
    auto signal = [&](int q) {
      fence_proxy_async_smem();  // these generic writes precede the next TMA write of the slot
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[q % S]);
    };
    // x and y ghosts of an in-domain plane (halo columns of every slot row, halo rows of every
    // slot column; the four halo corners are never read)
    auto fix_xy = [&](T* sx) {
      if (fxl || fxh)
        for (int r = lane; r < XH; r += 32) {
          T* row = sx + r * XW;
          if (fxl) {
            const T a0 = row[2], a1 = row[3], a2 = row[4], a3 = row[5];
            row[1] = ghost4<T>(txl, 0, a0, a1, a2, a3);
            row[0] = ghost4<T>(txl, 1, a0, a1, a2, a3);
          }
          if (fxh) {
            const T a0 = row[XW - 3], a1 = row[XW - 4], a2 = row[XW - 5], a3 = row[XW - 6];
            row[XW - 2] = ghost4<T>(txh, 0, a0, a1, a2, a3);
            row[XW - 1] = ghost4<T>(txh, 1, a0, a1, a2, a3);
          }
        }
      if (fyl || fyh)
        for (int c = lane + 2; c < XW - 2; c += 32) {
          if (fyl) {
            const T a0 = sx[2 * XW + c], a1 = sx[3 * XW + c], a2 = sx[4 * XW + c], a3 = sx[5 * XW + c];
            sx[1 * XW + c] = ghost4<T>(tyl, 0, a0, a1, a2, a3);
            sx[0 * XW + c] = ghost4<T>(tyl, 1, a0, a1, a2, a3);
          }
          if (fyh) {
            const T a0 = sx[(TY + 1) * XW + c], a1 = sx[TY * XW + c], a2 = sx[(TY - 1) * XW + c],
                    a3 = sx[(TY - 2) * XW + c];
            sx[(TY + 2) * XW + c] = ghost4<T>(tyh, 0, a0, a1, a2, a3);
            sx[(TY + 3) * XW + c] = ghost4<T>(tyh, 1, a0, a1, a2, a3);
          }
        }
    };
    // a z ghost plane (layer 0 or 1) over the tile's cells from four in-domain planes, the
    // first next to the face
    auto fix_z = [&](T* dst, int type, int layer, const T* b0, const T* b1, const T* b2, const T* b3) {
      for (int e = lane; e < TY * TX; e += 32) {
        const int o = (e / TX + 2) * XW + (e % TX) + 2;
        dst[o] = ghost4<T>(type, layer, b0[o], b1[o], b2[o], b3[o]);
      }
    };
    int q = 0;
    if (fzl) {
      // planes ka .. ka+3 first (they define the two ghost planes below the face)
      for (int t = 2; t < 6; ++t) {
        if (!wait_full(t)) { if (lane == 0) atomicOr(err, 1u); return; }
        fix_xy(slot(t));
      }
      for (int t = 0; t < 2; ++t) wait_full(t);  // plain arrivals: complete at once
      fix_z(slot(1), tzl, 0, slot(2), slot(3), slot(4), slot(5));
      fix_z(slot(0), tzl, 1, slot(2), slot(3), slot(4), slot(5));
      for (int t = 0; t < 6; ++t) signal(t);
      q = 6;
    }
    for (; q < np; ++q) {
      const int k = kfirst + q;
      if (!wait_full(q)) { if (lane == 0) atomicOr(err, 1u); return; }
      if (lz + k >= nzd) {
        // ghost planes above the face from planes nzd-1 .. nzd-4 (still in the ring: none of
        // their slots is reused before the chunk ends)
        const int layer = lz + k - nzd;
        const int qa = nzd - 1 - lz - kfirst;
        fix_z(slot(q), tzh, layer, slot(qa), slot(qa - 1), slot(qa - 2), slot(qa - 3));
      } else {
        fix_xy(slot(q));
      }
      signal(q);
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  unsigned long long* gbar = fix ? ready : full;  // block-uniform: the fixer's signal, or the copies'
  const T kc2 = beta * inv, kc1 = T(16) * kc2, kc0 = alpha - T(90) * kc2;
  const unsigned char* __restrict__ vb = (MODE == OP_RESID && vmask) ? vmask + p.off : nullptr;
  const int c0 = 2 + 2 * lane;  // slot column of the lane's first cell
  int wxy[RW][2];               // x + 5 y distance classes of the lane's cells
  {
    const int kx0 = face_class(gx0 + 2 * lane, lv.ndom[0]), kx1 = face_class(gx0 + 2 * lane + 1, lv.ndom[0]);
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int wy = 5 * face_class(gy0 + warp * RW + r, lv.ndom[1]);
      wxy[r][0] = kx0 + wy;
      wxy[r][1] = kx1 + wy;
    }
  }
  auto fail = [&]() {
    if (lane == 0) atomicOr(err, 1u);
  };
  // output of the lane's first cell, first row, plane ka (patch-relative, then advanced by sz)
  T* __restrict__ orow = out + p.off + (long long)(ka + NG) * p.sz + (long long)(j0 + NG + warp * RW) * p.sy + (i0 + c0);
  const unsigned char* __restrict__ vrow =
      vb ? vb + (long long)(ka + NG) * p.sz + (long long)(j0 + NG + warp * RW) * p.sy + (i0 + c0) : nullptr;
  const int sy = (int)p.sy, sz = (int)p.sz;

  if constexpr (!NEEDX) {
    // first sweep from x = 0: out = w f, plane by plane
    for (int k = ka, q = 0; k < kb; ++k, ++q) {
      if (!mbar_wait(&full[q % S], (unsigned)((q / S) & 1))) { fail(); return; }
      const T* sf = ring + (size_t)(q % S) * SLOT;
      const int kz25 = 25 * face_class(lz + k, nzd);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const V fk = ld2<T>(sf + (warp * RW + r) * XW + c0);
        st2<T>(orow + r * sy, V{wt[wxy[r][0] + kz25] * fk.x, wt[wxy[r][1] + kz25] * fk.y});
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[q % S]);
      orow += sz;
    }
    return;
  } else {
    // planes ka-2 .. ka+1 before the first step
    for (int q = 0; q < 4; ++q)
      if (!mbar_wait(&gbar[q], 0u)) { fail(); return; }
    const T* pz[5];  // slots of planes k-2 .. k+2
#pragma unroll
    for (int d = 0; d < 4; ++d) pz[d] = ring + (size_t)d * SLOT;
    int s4 = 4, par4 = 0;  // slot and phase parity of plane k+2
    const int rbase = (warp * RW + 2) * XW + c0;
    // f of the lane's pairs, loaded two planes ahead into two register slots used alternately
    // (no register with a load in flight is copied)
    const T* __restrict__ frow =
        NEEDF ? f + p.off + (long long)(ka + NG) * p.sz + (long long)(j0 + NG + warp * RW) * p.sy + (i0 + c0) : nullptr;
    V fq[2][RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      fq[0][r] = fq[1][r] = V{T(0), T(0)};
      if (NEEDF) {
        fq[0][r] = __ldg(reinterpret_cast<const V*>(frow + r * sy));
        if (ka + 1 < kb) fq[1][r] = __ldg(reinterpret_cast<const V*>(frow + sz + r * sy));
      }
    }
    // the valid mask of the lane's pairs (masked residual), two planes ahead like f
    uchar2 mq[2][RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      mq[0][r] = mq[1][r] = make_uchar2(1, 1);
      if (vrow != nullptr) {
        mq[0][r] = *reinterpret_cast<const uchar2*>(vrow + r * sy);
        if (ka + 1 < kb) mq[1][r] = *reinterpret_cast<const uchar2*>(vrow + sz + r * sy);
      }
    }
    // restriction: the coarse cell of the lane (x: its pair, y: the warp's two rows, z: a
    // plane pair) and the running sum of its children
    T racc = T(0);
    T* __restrict__ crow = nullptr;
    if (MODE == OP_RESTRICT)
      crow = outc + cpd.off + comp * ccs + (long long)((lz + ka) / 2 - cpd.lo[2] + NG) * cpd.sz +
             (long long)((gy0 + warp * RW) / 2 - cpd.lo[1] + NG) * cpd.sy + (gx0 / 2 + lane - cpd.lo[0] + NG);
    auto step = [&](int k, auto slotc) -> bool {
      constexpr int FS = decltype(slotc)::value;
      pz[4] = ring + (size_t)s4 * SLOT;
      if (!mbar_wait(&gbar[s4], (unsigned)par4)) return false;
      const T* __restrict__ sx = pz[2];
      const int kz25 = 25 * face_class(lz + k, nzd);
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        const int sr = rbase + r * XW;
        const V xc = ld2<T>(sx + sr);
        const V xl = ld2<T>(sx + sr - 2), xr = ld2<T>(sx + sr + 2);
        const V ym1 = ld2<T>(sx + sr - XW), ym2 = ld2<T>(sx + sr - 2 * XW);
        const V yp1 = ld2<T>(sx + sr + XW), yp2 = ld2<T>(sx + sr + 2 * XW);
        const V zm2 = ld2<T>(pz[0] + sr), zm1 = ld2<T>(pz[1] + sr);
        const V zp1 = ld2<T>(pz[3] + sr), zp2 = ld2<T>(pz[4] + sr);
        // cell 0 of the pair: x neighbours xl.y (-1), xl.x (-2), xc.y (+1), xr.x (+2);
        // cell 1: xc.x (-1), xl.y (-2), xr.x (+1), xr.y (+2)
        const T s1a = ((xl.y + xc.y) + (ym1.x + yp1.x)) + (zm1.x + zp1.x);
        const T s2a = ((xl.x + xr.x) + (ym2.x + yp2.x)) + (zm2.x + zp2.x);
        const T s1b = ((xc.x + xr.x) + (ym1.y + yp1.y)) + (zm1.y + zp1.y);
        const T s2b = ((xl.y + xr.y) + (ym2.y + yp2.y)) + (zm2.y + zp2.y);
        T o0, o1;
        if (MODE == OP_RESTRICT) {
          // cell_Lx and cell_restrict: (16 s1 - s2 - 90 x) + 0, f - (alpha x + beta (s inv)),
          // children summed x fastest, then y, then z
          const V fk = fq[FS][r];
          if (k + 2 < kb) fq[FS][r] = __ldg(reinterpret_cast<const V*>(frow + 2 * sz + r * sy));
          const T sa = (T(16) * s1a - s2a - T(90) * xc.x) + T(0);
          const T sb = (T(16) * s1b - s2b - T(90) * xc.y) + T(0);
          racc += fk.x - (alpha * xc.x + beta * (sa * inv));
          racc += fk.y - (alpha * xc.y + beta * (sb * inv));
          continue;
        } else if (MODE == OP_APPLY) {
          o0 = kc0 * xc.x + (kc1 * s1a - kc2 * s2a);
          o1 = kc0 * xc.y + (kc1 * s1b - kc2 * s2b);
        } else {
          const V fk = fq[FS][r];
          if (k + 2 < kb) fq[FS][r] = __ldg(reinterpret_cast<const V*>(frow + 2 * sz + r * sy));
          const T ra = fma(kc2, s2a, fma(-kc1, s1a, fma(-kc0, xc.x, fk.x)));
          const T rb = fma(kc2, s2b, fma(-kc1, s1b, fma(-kc0, xc.y, fk.y)));
          if (MODE == OP_RESID) {
            o0 = ra;
            o1 = rb;
          } else {
            o0 = fma(wt[wxy[r][0] + kz25], ra, xc.x);
            o1 = fma(wt[wxy[r][1] + kz25], rb, xc.y);
          }
        }
        if (vrow != nullptr) {
          // the pair's two mask bytes in one load; both valid (everywhere outside the region a
          // finer level covers, and inside it both are invalid): one paired store
          const uchar2 vm = mq[FS][r];
          if (k + 2 < kb) mq[FS][r] = *reinterpret_cast<const uchar2*>(vrow + 2 * sz + r * sy);
          if (vm.x && vm.y) {
            st2<T>(orow + r * sy, V{o0, o1});
          } else {
            if (vm.x) orow[r * sy] = o0;
            if (vm.y) orow[r * sy + 1] = o1;
          }
        } else {
          st2<T>(orow + r * sy, V{o0, o1});
        }
      }
      if (MODE == OP_RESTRICT && ((k - ka) & 1)) {  // second plane of the pair: the coarse value
        *crow = racc * T(0.125);
        crow += cpd.sz;
        racc = T(0);
      }
      // plane k-2 is no longer read: release its slot
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[(pz[0] - ring) / SLOT]);
#pragma unroll
      for (int d = 0; d < 4; ++d) pz[d] = pz[d + 1];
      if (++s4 == S) {
        s4 = 0;
        par4 ^= 1;
      }
      orow += sz;
      if (vrow) vrow += sz;
      if (NEEDF) frow += sz;
      return true;
    };
    for (int k = ka; k < kb; k += 2) {
      if (!step(k, zc_slot<0>{})) { fail(); return; }
      if (k + 1 < kb && !step(k + 1, zc_slot<1>{})) { fail(); return; }
    }
  }
}


// ------------------------------------------------------------------ FP64 residual, fixed point
// The refinement loop's FP64 residual r = f - (alpha x + beta L x) on the same single-patch
// levels, with the stencil sums formed exactly in 64-bit integers as in k_resid3d_fx (frame:
// the level's largest interior |x|, found by k_absmax_patch, its leading bit at bit 52;
// T = 16 s1 - s2 - 90 x = 12 h^2 L x 2^S exact; r = f - alpha x - (beta / 12 h^2) 2^-S T by
// two FP64 multiply-adds).  The planes of x are streamed by the producer as in k_sweep3d;
// NFW converter warps then rewrite every staged value that the stencil reads as its
// fixed-point integer, in place (one conversion per staged value instead of one per read),
// write the physical ghost values of face tiles (x and y: from the converted cells next to
// the face, rounded to integers; z ghost planes: from the stored cells, rounded to the
// frame: the same values as k_resid3d_fx), and release the plane to the consumer warps,
// which read integer neighbour pairs from the ring, f from a second ring of SF slots (one
// plane of the tile per slot, also filled by the producer) and x itself (for alpha x) from
// global memory one plane ahead (the plane was just brought into L2 by the copy).
// The result is bit for bit that of k_resid3d_fx.  A value outside the frame sets the
// replica's flag (lv.fxs[2 c + 1]), and the plain FP64 kernel launched after this one
// recomputes the level.
template <int TY, int RW, int S, int NFW>
constexpr int rfx_threads() {
  return 32 * (TY / RW + 1 + NFW);
}
constexpr int RFX_SF = 3;  // slots of the f ring
template <int TY, int S>
constexpr size_t rfx_smem_bytes() {
  return ((size_t)S * sw3::region_elems<double>(TY + 4) + (size_t)RFX_SF * sw3::region_elems<double>(TY)) *
             sizeof(double) +
         (3 * S + 2 * RFX_SF) * sizeof(unsigned long long);
}

template <int TY, int RW, int S, int NFW>
__global__ void __launch_bounds__(rfx_threads<TY, RW, S, NFW>(), 2)
    k_resid3d_fx_tma(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmf, LevelView lv,
                     int ntx, int ntiles, int nch,
                     const double* __restrict__ x, const double* __restrict__ f, double* __restrict__ out,
                     double alpha, double beta) {
  using namespace sw3;
  unsigned* err = &g_sweep3d_err;
  constexpr int NCW = TY / RW;        // consumer warps
  constexpr int XH = TY + 4;          // slot rows
  constexpr int SLOT = region_elems<double>(XH);
  constexpr int SF = RFX_SF, FSLOT = region_elems<double>(TY);
  constexpr int NFT = 32 * NFW;       // converter threads
  constexpr int EPL = (XH * XW + NFT - 1) / NFT;  // staged values per converter thread
  static_assert(TY % RW == 0 && S >= 8 && EPL <= 32, "tile rows must split into warps; eight slots; mask width");
  extern __shared__ __align__(128) unsigned char sw3_smem[];
  long long* ring = reinterpret_cast<long long*>(sw3_smem);
  double* fring = reinterpret_cast<double*>(ring + (size_t)S * SLOT);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(fring + (size_t)SF * FSLOT);
  unsigned long long* ready = full + S;
  unsigned long long* empty = ready + S;
  unsigned long long* ffull = empty + S;
  unsigned long long* fempty = ffull + SF;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bpc = gridDim.x / lv.ncomp, comp = blockIdx.x / bpc, blk = blockIdx.x % bpc;
  PatchDesc p = lv.p0;
  p.off += comp * lv.cstride;
  const int nz = p.n[2];
  const int tile = blk % ntiles, chunk = blk / ntiles;
  const int ka = (int)(((long long)chunk * nz) / nch), kb = (int)(((long long)(chunk + 1) * nz) / nch);
  const int i0 = (tile % ntx) * TX, j0 = (tile / ntx) * TY;
  const int lz = p.lo[2], nzd = lv.ndom[2];
  const int gx0 = p.lo[0] + i0, gy0 = p.lo[1] + j0;
  const bool fxl = gx0 == 0, fxh = gx0 + TX == lv.ndom[0], fyl = gy0 == 0, fyh = gy0 + TY == lv.ndom[1];
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&ready[q], NFW);
      mbar_init(&empty[q], NCW);
    }
    for (int q = 0; q < SF; ++q) {
      mbar_init(&ffull[q], 1);
      mbar_init(&fempty[q], NCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (ka >= kb) return;
  pdl_wait();  // the frame is written by the preceding kernel
  if (lv.active != nullptr && !lv.active[comp]) return;  // converged replica of a stacked batch
  unsigned* __restrict__ flag = reinterpret_cast<unsigned*>(lv.fxs + 2 * comp + 1);
  const int emax = (int)((lv.fxs[2 * comp] >> 52) & 0x7ffull);
  if (emax == 0x7ff || (emax != 0 && emax < 53)) {  // non-finite, or a frame below the normal range
    if (tid == 0) *flag = 1u;
    return;
  }
  const int kfirst = ka - 2;
  const int np = (kb - ka) + 4;  // planes through the ring
  const int sy = (int)p.sy, sz = (int)p.sz;

  if (warp == NCW) {
    // ---------------------------------------------------------------- producer (one thread)
    // x plane q and, from q = 4 on, f plane q - 4 (the plane the consumers take when x plane q
    // completes their window)
    if (lane != 0) return;
    tma_prefetch_desc(&tmx);
    tma_prefetch_desc(&tmf);
    int q = 0, nf = 0;  // x planes and f planes issued
    bool ok = true;
    for (; q < np; ++q) {
      const int sl = q % S, use = q / S, k = kfirst + q;
      if (use > 0 && !mbar_wait(&empty[sl], (unsigned)((use - 1) & 1))) {
        ok = false;
        break;
      }
      if (lz + k < 0 || lz + k >= nzd) {  // z ghost plane: the converters write it
        mbar_arrive(&full[sl]);
      } else {
        mbar_expect_tx(&full[sl], (unsigned)(XH * XW * sizeof(double)));
        tma_load4(ring + (size_t)sl * SLOT, &tmx, i0, j0, k + NG, comp, &full[sl]);
      }
      const int j = q - 4;
      if (j >= 0) {
        const int fs = j % SF, fuse = j / SF;
        if (fuse > 0 && !mbar_wait(&fempty[fs], (unsigned)((fuse - 1) & 1))) {
          ok = false;
          ++q;  // x plane q was issued
          break;
        }
        mbar_expect_tx(&ffull[fs], (unsigned)(TY * XW * sizeof(double)));
        tma_load4(fring + (size_t)fs * FSLOT, &tmf, i0, j0 + NG, ka + j + NG, comp, &ffull[fs]);
        ++nf;
      }
    }
    if (!ok) atomicOr(err, 1u);
    // the block must not end while copies into its shared memory are in flight: wait
    // (bounded) for the last copies issued into every slot of both rings
    for (int t = max(0, q - S); t < q; ++t) mbar_wait(&full[t % S], (unsigned)((t / S) & 1));
    for (int t = max(0, nf - SF); t < nf; ++t) mbar_wait(&ffull[t % SF], (unsigned)((t / SF) & 1));
    return;
  }

  if (warp > NCW) {
    // ---------------------------------------------------------------- converters (NFW warps)
    const int ft = tid - 32 * (NCW + 1);
    bool ovf = false;
    // staged values this thread converts (bit t: value ft + t NFT): not a halo corner (never
    // read) and not a physical ghost (written from the converted cells afterwards)
    unsigned cmask = 0u;
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
      const int e = ft + t * NFT;
      if (e >= XH * XW) continue;
      const int r = e / XW, c = e % XW;
      const bool hr = r < 2 || r >= TY + 2, hc = c < 2 || c >= TX + 2;
      const bool ghost = (c < 2 && fxl) || (c >= TX + 2 && fxh) || (r < 2 && fyl) || (r >= TY + 2 && fyh);
      if (!(hr && hc) && !ghost) cmask |= 1u << t;
    }
    auto fbar = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(NFT) : "memory"); };
    auto slot = [&](int q) -> long long* { return ring + (size_t)(q % S) * SLOT; };
    // physical ghost value of layer ``layer`` from four converted cells (below 2^53: exact
    // as FP64), already in frame units, rounded to an integer
    auto gfx = [&](int type, int layer, long long a0, long long a1, long long a2, long long a3) -> long long {
      const double v = ghost4<double>(type, layer, (double)a0, (double)a1, (double)a2, (double)a3);
      return fx_of(v, 1075, 7, ovf);
    };
    const bool fxy = fxl || fxh || fyl || fyh;  // block-uniform
    const double* __restrict__ xb = x + p.off;
    // Every converter warp passes the same sequence of converter barriers (their number
    // depends on block-uniform values only), also after a wait ran out: then it skips the
    // work and the remaining waits, so that no barrier is left waiting for it.
    bool ok = true;
    for (int q = 0; q < np; ++q) {
      const int k = kfirst + q, g = lz + k;
      long long* sq = slot(q);
      ok = ok && mbar_wait(&full[q % S], (unsigned)((q / S) & 1));
      if (g < 0 || g >= nzd) {
        // z ghost plane over the tile's cells from the four stored planes next to the face
        // (global memory), rounded to the frame
        if (ok) {
          const int side = g < 0 ? 0 : 1, layer = side == 0 ? -g - 1 : g - nzd, type = lv.bc[4 + side];
          const int k0 = (side == 0 ? 0 : nzd - 1) - lz + NG, dk = side == 0 ? sz : -sz;
          for (int e = ft; e < TY * TX; e += NFT) {
            const int ii = e % TX, jj = e / TX;
            const double* col = xb + (long long)k0 * sz + (long long)(j0 + jj + NG) * sy + (i0 + ii + NG);
            const double v = ghost4<double>(type, layer, col[0], col[dk], col[2 * dk], col[3 * dk]);
            sq[(jj + 2) * XW + ii + 2] = fx_of(v, emax, 7, ovf);
          }
        }
      } else {
        if (ok) {
          // stored values to integers, in place (each thread rewrites only its own values)
          const double* sd = reinterpret_cast<const double*>(sq);
#pragma unroll
          for (int t = 0; t < EPL; ++t)
            if ((cmask >> t) & 1u) {
              const int e = ft + t * NFT;
              sq[e] = fx_of(sd[e], emax, 2, ovf);
            }
        }
        if (fxy) {
          fbar();  // every converter's cells of this plane are integers
          if (ok) {
            // x and y ghosts (rows / columns of the tile's cells only: the halo corners are
            // never read)
            const int txl = lv.bc[0], txh = lv.bc[1], tyl = lv.bc[2], tyh = lv.bc[3];
            if (fxl || fxh)
              for (int r = ft + 2; r < TY + 2; r += NFT) {
                long long* row = sq + r * XW;
                if (fxl) {
                  const long long a0 = row[2], a1 = row[3], a2 = row[4], a3 = row[5];
                  row[1] = gfx(txl, 0, a0, a1, a2, a3);
                  row[0] = gfx(txl, 1, a0, a1, a2, a3);
                }
                if (fxh) {
                  const long long a0 = row[XW - 3], a1 = row[XW - 4], a2 = row[XW - 5], a3 = row[XW - 6];
                  row[XW - 2] = gfx(txh, 0, a0, a1, a2, a3);
                  row[XW - 1] = gfx(txh, 1, a0, a1, a2, a3);
                }
              }
            if (fyl || fyh)
              for (int c = ft + 2; c < XW - 2; c += NFT) {
                if (fyl) {
                  const long long a0 = sq[2 * XW + c], a1 = sq[3 * XW + c], a2 = sq[4 * XW + c], a3 = sq[5 * XW + c];
                  sq[1 * XW + c] = gfx(tyl, 0, a0, a1, a2, a3);
                  sq[0 * XW + c] = gfx(tyl, 1, a0, a1, a2, a3);
                }
                if (fyh) {
                  const long long a0 = sq[(TY + 1) * XW + c], a1 = sq[TY * XW + c], a2 = sq[(TY - 1) * XW + c],
                                  a3 = sq[(TY - 2) * XW + c];
                  sq[(TY + 2) * XW + c] = gfx(tyh, 0, a0, a1, a2, a3);
                  sq[(TY + 3) * XW + c] = gfx(tyh, 1, a0, a1, a2, a3);
                }
              }
          }
        }
      }
      fence_proxy_async_smem();  // these generic writes precede the next TMA write of the slot
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[q % S]);
    }
    if (!ok && lane == 0) atomicOr(err, 1u);
    if (ovf) *flag = 1u;
    return;
  }

  // ------------------------------------------------------------------ consumers
  using L2v = longlong2;
  const double kT = emax == 0 ? 0.0 : beta * lv.inv12h2 * __longlong_as_double((long long)(emax - 52) << 52);
  const bool has_a = alpha != 0.0;  // block-uniform
  const int c0 = 2 + 2 * lane;
  const long long o0 = p.off + (long long)(ka + NG) * p.sz + (long long)(j0 + NG + warp * RW) * p.sy + (i0 + c0);
  double* __restrict__ orow = out + o0;
  const double* __restrict__ xrow = x + o0;
  auto fail = [&]() {
    if (lane == 0) atomicOr(err, 1u);
  };
  for (int q = 0; q < 4; ++q)
    if (!mbar_wait(&ready[q], 0u)) { fail(); return; }
  const long long* pz[5];
#pragma unroll
  for (int d = 0; d < 4; ++d) pz[d] = ring + (size_t)d * SLOT;
  int s4 = 4, par4 = 0, fs = 0, fpar = 0;
  const int rbase = (warp * RW + 2) * XW + c0;
  const int fbase = warp * RW * XW + c0;
  double2 xq[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) xq[r] = has_a ? *reinterpret_cast<const double2*>(xrow + r * sy) : make_double2(0.0, 0.0);
  for (int k = ka; k < kb; ++k) {
    pz[4] = ring + (size_t)s4 * SLOT;
    if (!mbar_wait(&ready[s4], (unsigned)par4) || !mbar_wait(&ffull[fs], (unsigned)fpar)) { fail(); return; }
    const long long* __restrict__ sx = pz[2];
    const double* __restrict__ sf = fring + (size_t)fs * FSLOT;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int sr = rbase + r * XW;
      const L2v xc = *reinterpret_cast<const L2v*>(sx + sr);
      const L2v xl = *reinterpret_cast<const L2v*>(sx + sr - 2), xr = *reinterpret_cast<const L2v*>(sx + sr + 2);
      const L2v ym1 = *reinterpret_cast<const L2v*>(sx + sr - XW), ym2 = *reinterpret_cast<const L2v*>(sx + sr - 2 * XW);
      const L2v yp1 = *reinterpret_cast<const L2v*>(sx + sr + XW), yp2 = *reinterpret_cast<const L2v*>(sx + sr + 2 * XW);
      const L2v zm2 = *reinterpret_cast<const L2v*>(pz[0] + sr), zm1 = *reinterpret_cast<const L2v*>(pz[1] + sr);
      const L2v zp1 = *reinterpret_cast<const L2v*>(pz[3] + sr), zp2 = *reinterpret_cast<const L2v*>(pz[4] + sr);
      // cell 0 of the pair: x neighbours xl.y (-1), xl.x (-2), xc.y (+1), xr.x (+2);
      // cell 1: xc.x (-1), xl.y (-2), xr.x (+1), xr.y (+2)
      const long long s1a = ((xl.y + xc.y) + (ym1.x + yp1.x)) + (zm1.x + zp1.x);
      const long long s2a = ((xl.x + xr.x) + (ym2.x + yp2.x)) + (zm2.x + zp2.x);
      const long long s1b = ((xc.x + xr.x) + (ym1.y + yp1.y)) + (zm1.y + zp1.y);
      const long long s2b = ((xl.y + xr.y) + (ym2.y + yp2.y)) + (zm2.y + zp2.y);
      const long long Ta = s1a * 16 - s2a - xc.x * 90;
      const long long Tb = s1b * 16 - s2b - xc.y * 90;
      const double2 fk = *reinterpret_cast<const double2*>(sf + fbase + r * XW);
      const double2 xk = xq[r];
      if (has_a && k + 1 < kb) xq[r] = *reinterpret_cast<const double2*>(xrow + sz + r * sy);
      // (alpha = 0, the pressure Poisson equation: f - 0 x is f, one FP64 operation per cell)
      const double ra = fma(-kT, fx_to_double(Ta), has_a ? fma(-alpha, xk.x, fk.x) : fk.x);
      const double rb = fma(-kT, fx_to_double(Tb), has_a ? fma(-alpha, xk.y, fk.y) : fk.y);
      *reinterpret_cast<double2*>(orow + r * sy) = make_double2(ra, rb);
    }
    // plane k-2 of x and plane k of f are no longer read: release their slots
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[(pz[0] - ring) / SLOT]);
      mbar_arrive(&fempty[fs]);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) pz[d] = pz[d + 1];
    if (++s4 == S) {
      s4 = 0;
      par4 ^= 1;
    }
    if (++fs == SF) {
      fs = 0;
      fpar ^= 1;
    }
    orow += sz;
    xrow += sz;
  }
}

}  // namespace amr4
