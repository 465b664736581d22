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


// ------------------------------------------------------------------ cube coarse V-cycle
// The coarse end of a 3-D level-0 pyramid N0^3, (N0/2)^3, ... down to the bottom grid, in one
// block of 1024 threads with every grid in shared memory and every size a compile-time
// constant (the 3-D counterpart of k_mg_coarse2d_sq; FP32: N0 = 16, grids 16, 8 and the 4^3
// bottom).  Same V-cycle as the per-grid kernels: nu1 weighted-Jacobi sweeps (the first from
// zero), residual restriction (mean of the eight children), the dense bottom solve, linear
// prolongation of the correction with the homogeneous extension of the coarse values beyond
// the domain (applied dimension after dimension, edges and corners included), nu2 sweeps.
// Before a sweep reads an array, one pass writes its two physical ghost layers on the six
// faces (Eqs. velBCHomoDiri5th, Neumann5); the 13-point stencil never reads edges or corners.
constexpr int CU_NT = 1024;

template <int N>
struct Cu {
  static constexpr int S = N + 4;     // row pitch
  static constexpr int P = S * S;     // plane pitch
  static constexpr int E = P * S;     // elements of one array
  static constexpr bool bottom = (N % 2 != 0) || (N / 2 < MIN_BOX);
};
template <int N0, int N>
__host__ __device__ constexpr int cu_off() {
  if constexpr (N >= N0) return 0;
  else return cu_off<N0, 2 * N>() + 3 * Cu<2 * N>::E;
}
template <int N0, int N>
__host__ __device__ constexpr int cu_total() {
  if constexpr (Cu<N>::bottom) return cu_off<N0, N>() + 3 * Cu<N>::E;
  else return cu_total<N0, N / 2>();
}
template <int N0, int N>
__host__ __device__ constexpr int cu_bottom() {
  if constexpr (Cu<N>::bottom) return N;
  else return cu_bottom<N0, N / 2>();
}
template <int N0, int N>
__host__ __device__ constexpr int cu_depth() {
  if constexpr (N >= N0) return 0;
  else return 1 + cu_depth<N0, 2 * N>();
}
template <int N0>
__host__ __device__ constexpr int cu_ngrids() {
  return 1 + cu_depth<N0, cu_bottom<N0, N0>()>();
}

struct CubeBlock {
  int nu1, nu2;
  int nbot, ldb;
  int bcm;              // boundary type of face f (0 Dirichlet, 1 Neumann) in bit f
  const double* minv;   // bottom inverse
  PatchDesc gp;         // global layout of the top grid (right-hand side in, correction out)
  float wt[4][125];     // omega / diag per grid and distance class kx + 5 ky + 25 kz
  float binv[4];        // beta / (12 h^2) per grid
  float alpha;
  long long cstride;    // stacked component batches: replica stride of the top grid's arrays
  const int* active;    // and the replicas still iterating (null for one replica)
};

template <typename T, int N0>
struct CubeVcycle {
  T* sm;
  const CubeBlock* cb;
  double* bot;
  template <int N> __device__ T* X() const { return sm + cu_off<N0, N>(); }
  template <int N> __device__ T* Tt() const { return sm + cu_off<N0, N>() + Cu<N>::E; }
  template <int N> __device__ T* B() const { return sm + cu_off<N0, N>() + 2 * Cu<N>::E; }
  __device__ static int tid() { return threadIdx.x + 32 * threadIdx.y; }
  __device__ int bc(int f) const { return (cb->bcm >> f) & 1; }
  template <int N> __device__ static int at(int i, int j, int k) {
    return (k + 2) * Cu<N>::P + (j + 2) * Cu<N>::S + i + 2;
  }

  // the two physical ghost layers of the six faces (face cells only), from the four cells
  // next to each face
  template <int N>
  __device__ void ghosts(T* a) const {
    constexpr int NE = 12 * N * N, IT = (NE + CU_NT - 1) / CU_NT;
    const int st[3] = {1, Cu<N>::S, Cu<N>::P};
#pragma unroll
    for (int q = 0; q < IT; ++q) {
      const int e = tid() + q * CU_NT;
      if (NE % CU_NT == 0 || e < NE) {
        const int f = e / (2 * N * N), r = e % (2 * N * N), layer = r & 1, pos = r >> 1;
        const int d = f >> 1, side = f & 1, t = bc(f);
        const int u = pos % N, v = pos / N;  // the two other coordinates, lower dimension first
        int c[3];
        c[d] = side == 0 ? 0 : N - 1;
        c[d == 0 ? 1 : 0] = u;
        c[d == 2 ? 1 : 2] = v;
        const int o = at<N>(c[0], c[1], c[2]);
        const int in = side == 0 ? st[d] : -st[d];  // towards the interior
        T g = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) g += gcoef<T>(t, layer, m) * a[o + m * in];
        a[o - (layer + 1) * in] = g;
      }
    }
    __syncthreads();
  }

  // layer-1 extension of a coarse correction beyond the domain, dimension after dimension
  // (x over the interior rows, y over rows extended in x, z over planes extended in x and y)
  template <int N>
  __device__ void extend(T* a) const {
    const int st[3] = {1, Cu<N>::S, Cu<N>::P};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // the other two coordinates run over -1 .. N where already extended, else 0 .. N-1
      const int n1 = d >= 1 ? N + 2 : N, n2 = d >= 2 ? N + 2 : N;
      const int NE = 2 * n1 * n2;
      for (int e = tid(); e < NE; e += CU_NT) {
        const int side = e & 1, pos = e >> 1;
        const int u = pos % n1 - (d >= 1 ? 1 : 0), v = pos / n1 - (d >= 2 ? 1 : 0);
        int c[3];
        c[d] = side == 0 ? 0 : N - 1;
        c[d == 0 ? 1 : 0] = u;
        c[d == 2 ? 1 : 2] = v;
        const int o = at<N>(c[0], c[1], c[2]);
        const int in = side == 0 ? st[d] : -st[d];
        const int t = bc(2 * d + side);
        T g = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) g += gcoef<T>(t, 0, m) * a[o + m * in];
        a[o - in] = g;
      }
      __syncthreads();
    }
  }

  template <int N>
  __device__ static T ax(const T* __restrict__ a, int o, T alpha, T binv) {
    constexpr int S = Cu<N>::S, P = Cu<N>::P;
    const T xc = a[o];
    const T s1 = ((a[o - 1] + a[o + 1]) + (a[o - S] + a[o + S])) + (a[o - P] + a[o + P]);
    const T s2 = ((a[o - 2] + a[o + 2]) + (a[o - 2 * S] + a[o + 2 * S])) + (a[o - 2 * P] + a[o + 2 * P]);
    return alpha * xc + binv * ((T(16) * s1 - s2 - T(90) * xc) + T(0));
  }

  template <int N>
  __device__ T* smooth(T* a, T* o, int nu, bool zero) const {
    constexpr int NC = N * N * N, IT = (NC + CU_NT - 1) / CU_NT;
    const T* b = B<N>();
    const float* w = cb->wt[cu_depth<N0, N>()];
    const T bi = T(cb->binv[cu_depth<N0, N>()]), al = T(cb->alpha);
    for (int s = 0; s < nu; ++s) {
      const bool z = zero && s == 0;
      if (!z) ghosts<N>(a);
#pragma unroll
      for (int q = 0; q < IT; ++q) {
        const int cidx = tid() + q * CU_NT;
        if (NC % CU_NT == 0 || cidx < NC) {
          const int i = cidx % N, j = (cidx / N) % N, k = cidx / (N * N);
          const int oc = at<N>(i, j, k);
          const T wc = T(w[face_class(i, N) + 5 * face_class(j, N) + 25 * face_class(k, N)]);
          if (z) a[oc] = wc * b[oc];
          else o[oc] = a[oc] + wc * (b[oc] - ax<N>(a, oc, al, bi));
        }
      }
      __syncthreads();
      if (!z) { T* sw = a; a = o; o = sw; }
    }
    return a;
  }

  template <int N>
  __device__ void restrict_residual(T* a) const {
    constexpr int M = N / 2, NC = M * M * M, IT = (NC + CU_NT - 1) / CU_NT;
    const T* b = B<N>();
    T* bc_ = B<M>();
    const T bi = T(cb->binv[cu_depth<N0, N>()]), al = T(cb->alpha);
    ghosts<N>(a);
#pragma unroll
    for (int q = 0; q < IT; ++q) {
      const int cidx = tid() + q * CU_NT;
      if (NC % CU_NT == 0 || cidx < NC) {
        const int ci = cidx % M, cj = (cidx / M) % M, ck = cidx / (M * M);
        T acc = T(0);
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
          for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
            for (int q0 = 0; q0 < 2; ++q0) {
              const int o = at<N>(2 * ci + q0, 2 * cj + q1, 2 * ck + q2);
              acc += b[o] - ax<N>(a, o, al, bi);
            }
        bc_[at<M>(ci, cj, ck)] = acc * T(0.125);
      }
    }
    __syncthreads();
  }

  template <int N>
  __device__ void prolong(T* a, T* cg) const {
    constexpr int M = N / 2, NC = N * N * N, IT = (NC + CU_NT - 1) / CU_NT;
    extend<M>(cg);
#pragma unroll
    for (int q = 0; q < IT; ++q) {
      const int cidx = tid() + q * CU_NT;
      if (NC % CU_NT == 0 || cidx < NC) {
        const int i = cidx % N, j = (cidx / N) % N, k = cidx / (N * N);
        const int oc = at<M>(i >> 1, j >> 1, k >> 1);
        const int d0 = (i & 1) ? 1 : -1, d1 = (j & 1) ? Cu<M>::S : -Cu<M>::S, d2 = (k & 1) ? Cu<M>::P : -Cu<M>::P;
        T v = T(0);
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
          for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
            for (int q0 = 0; q0 < 2; ++q0) {
              const T w = ((T(1) * (q0 == 0 ? T(0.75) : T(0.25))) * (q1 == 0 ? T(0.75) : T(0.25))) *
                          (q2 == 0 ? T(0.75) : T(0.25));
              v += w * cg[oc + q2 * d2 + q1 * d1 + q0 * d0];
            }
        a[at<N>(i, j, k)] += v;
      }
    }
    __syncthreads();
  }

  template <int N>
  __device__ void bottom() const {
    const T* b = B<N>();
    const int nb = cb->nbot;
    for (int t = tid(); t < nb; t += CU_NT) bot[t] = (double)b[at<N>(t % N, (t / N) % N, t / (N * N))];
    __syncthreads();
    T* x = X<N>();
    for (int t = tid(); t < nb; t += CU_NT) {
      double acc = 0.0;
      const double* row = cb->minv + (long long)t * cb->ldb;
      for (int c = 0; c < nb; ++c) acc = fma(row[c], bot[c], acc);
      x[at<N>(t % N, (t / N) % N, t / (N * N))] = T(acc);
    }
    __syncthreads();
  }

  template <int N>
  __device__ T* cycle() const {
    if constexpr (Cu<N>::bottom) {
      bottom<N>();
      return X<N>();
    } else {
      T* cur = smooth<N>(X<N>(), Tt<N>(), cb->nu1, true);
      restrict_residual<N>(cur);
      T* cg = cycle<N / 2>();
      prolong<N>(cur, cg);
      return smooth<N>(cur, cur == X<N>() ? Tt<N>() : X<N>(), cb->nu2, false);
    }
  }
};

template <typename T, int N0>
__global__ void __launch_bounds__(CU_NT) k_mg_coarse3d_cube(const __grid_constant__ CubeBlock cb,
                                                            const T* __restrict__ b, T* __restrict__ x) {
  pdl_wait();
  // stacked component batches: block c works on replica c (converged replicas return)
  const int rep = blockIdx.x;
  if (cb.active != nullptr && !cb.active[rep]) return;
  extern __shared__ __align__(16) unsigned char cu_smraw[];
  __shared__ double bot[Cu<cu_bottom<N0, N0>()>::E];
  CubeVcycle<T, N0> v;
  v.sm = reinterpret_cast<T*>(cu_smraw);
  v.cb = &cb;
  v.bot = bot;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  {
    const T* __restrict__ bg = b + cb.gp.off + rep * cb.cstride;
    T* bs = v.template B<N0>();
    for (int t = tid; t < N0 * N0 * N0; t += CU_NT) {
      const int i = t % N0, j = (t / N0) % N0, k = t / (N0 * N0);
      bs[CubeVcycle<T, N0>::template at<N0>(i, j, k)] = bg[(k + NG) * cb.gp.sz + (j + NG) * cb.gp.sy + i + NG];
    }
  }
  __syncthreads();
  const T* res = v.template cycle<N0>();
  T* __restrict__ xg = x + cb.gp.off + rep * cb.cstride;
  for (int t = tid; t < N0 * N0 * N0; t += CU_NT) {
    const int i = t % N0, j = (t / N0) % N0, k = t / (N0 * N0);
    xg[(k + NG) * cb.gp.sz + (j + NG) * cb.gp.sy + i + NG] = res[CubeVcycle<T, N0>::template at<N0>(i, j, k)];
  }
}

}  // namespace amr4
