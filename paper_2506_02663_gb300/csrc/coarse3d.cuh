// coarse3d.cuh -- the coarse end of a 3-D level-0 multigrid in one thread-block cluster.
//
// On the grids of 32^3 cells and fewer every kernel of a V-cycle (weighted-Jacobi sweeps,
// residual restriction, prolongation, the dense bottom solve of Sec. 6.5) runs in a few
// microseconds of launch latency and almost no work.  Here the whole coarse end -- the down
// legs, the bottom solve and the up legs of the grids m0 .. M -- is one launch of one
// cluster of CTAs (16 where the part allows it, else 8) that splits every phase's cells
// over all of its threads and separates the phases by hardware cluster barriers (release /
// acquire at cluster scope, which orders the global-memory writes of one phase before the
// reads of the next).  The per-cell arithmetic is the same device code as the per-grid
// kernels (cell_level_op, cell_restrict, cell_prolong, the bottom inverse), on the same
// global arrays, so the result is that of the per-grid launches.
#pragma once

#include "kernels.cuh"

namespace amr4 {

constexpr int CC_MAX = 6;            // grids of one cluster V-cycle
constexpr int CC_THREADS = 1024;     // threads per CTA
constexpr long long CC_CELLS = 32768;  // largest grid the cluster takes (32^3)

struct CoarseCluster {
  int ng;  // grids m0 .. m0 + ng - 1 (the last one is the bottom grid)
  int nu1, nu2;
  int nbot, ldb;
  const double* minv;          // bottom inverse (transposed for adjoint cycles)
  LevelView lv[CC_MAX];        // per-grid constants
  PatchDesc gp[CC_MAX];        // layout of each grid's arrays
};

template <typename T>
struct CoarsePtrs {
  T* x[CC_MAX];
  T* b[CC_MAX];
  T* t[CC_MAX];
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename T, int D, bool TR = false>
__global__ void __launch_bounds__(CC_THREADS) k_coarse_cluster(CoarseCluster cm, CoarsePtrs<T> ptr, T alpha, T beta,
                                                               T omega) {
  pdl_wait();
  unsigned rank, nranks;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(nranks));
  const int tid = (int)rank * blockDim.x + threadIdx.x, nth = (int)nranks * blockDim.x;
  auto ncell = [&](int m) { return cm.gp[m].n[0] * cm.gp[m].n[1] * cm.gp[m].n[2]; };
  int i, j, k;
  // down legs: nu1 sweeps from zero (the result ends in x), residual restricted into b[m+1]
  for (int m = 0; m + 1 < cm.ng; ++m) {
    T* x = ptr.x[m];
    T* tb = ptr.t[m];
    const T* b = ptr.b[m];
    T* cur = (cm.nu1 % 2 == 1) ? x : tb;
    T* oth = (cur == x) ? tb : x;
    for (int t = tid; t < ncell(m); t += nth) {
      cell_of(cm.gp[m], t, i, j, k);
      cell_level_op<T, D, OP_JACOBI0, TR>(cm.lv[m], cm.gp[m], i, j, k, nullptr, b, cur, nullptr, alpha, beta, omega);
    }
    cluster_barrier();
    for (int s = 1; s < cm.nu1; ++s) {
      for (int t = tid; t < ncell(m); t += nth) {
        cell_of(cm.gp[m], t, i, j, k);
        cell_level_op<T, D, OP_JACOBI, TR>(cm.lv[m], cm.gp[m], i, j, k, cur, b, oth, nullptr, alpha, beta, omega);
      }
      cluster_barrier();
      T* sw = cur;
      cur = oth;
      oth = sw;
    }
    for (int t = tid; t < ncell(m + 1); t += nth) {
      cell_of(cm.gp[m + 1], t, i, j, k);
      const int g[3] = {i, j, k};
      cell_restrict<T, D, true, TR>(cm.lv[m], cm.gp[m], cm.gp[m + 1], g, x, b, ptr.b[m + 1], alpha, beta);
    }
    cluster_barrier();
  }
  {
    // bottom: x = Minv b (the leading block of the bordered inverse for pure Neumann)
    const int M = cm.ng - 1;
    const T* b = ptr.b[M];
    T* x = ptr.x[M];
    for (int r = tid; r < cm.nbot; r += nth) {
      double acc = 0.0;
      const double* row = cm.minv + (long long)r * cm.ldb;
      for (int q = 0; q < cm.nbot; ++q) {
        cell_of(cm.gp[M], q, i, j, k);
        acc = fma(row[q], (double)b[poff(cm.gp[M], i, j, k)], acc);
      }
      cell_of(cm.gp[M], r, i, j, k);
      x[poff(cm.gp[M], i, j, k)] = T(acc);
    }
    cluster_barrier();
  }
  // up legs: prolongation of the coarse correction added to x, nu2 sweeps
  for (int m = cm.ng - 2; m >= 0; --m) {
    T* x = ptr.x[m];
    T* tb = ptr.t[m];
    const T* b = ptr.b[m];
    for (int t = tid; t < ncell(m); t += nth) {
      cell_of(cm.gp[m], t, i, j, k);
      const int gf[3] = {i, j, k};
      cell_prolong<T, D>(cm.lv[m + 1], cm.gp[m], cm.gp[m + 1], gf, ptr.x[m + 1], x, (T*)nullptr);
    }
    cluster_barrier();
    T* cur = x;
    T* oth = tb;
    for (int s = 0; s < cm.nu2; ++s) {
      for (int t = tid; t < ncell(m); t += nth) {
        cell_of(cm.gp[m], t, i, j, k);
        cell_level_op<T, D, OP_JACOBI, TR>(cm.lv[m], cm.gp[m], i, j, k, cur, b, oth, nullptr, alpha, beta, omega);
      }
      cluster_barrier();
      T* sw = cur;
      cur = oth;
      oth = sw;
    }
    if (cur != x) {
      for (int t = tid; t < ncell(m); t += nth) {
        cell_of(cm.gp[m], t, i, j, k);
        const long long o = poff(cm.gp[m], i, j, k);
        x[o] = cur[o];
      }
      cluster_barrier();
    }
  }
}

}  // namespace amr4
