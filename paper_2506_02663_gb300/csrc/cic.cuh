// Coarse-fine interface conditions of a subcycled level solve (Sec. 6.3, steps CIC-2 and
// CIC-3; Sec. 6.4, Eq. correctingFaceAvg).
//
//   k_cic_grp / k_cic   the CF ghost cells of level l at an intermediate time t*: AMRCFI of the
//                       level-(l-1) data at four equispaced coarse times, combined by the 2 x 4
//                       matrix I^(4)(k, eta) of Eq. (timeInterp) into the value at t* and its
//                       time derivative.  Both maps are linear, so each thread first forms the
//                       two time combinations of every coarse window cell and then applies the
//                       AMRCFI weights to them: one pass over the four windows and twice the
//                       AMRCFI arithmetic, instead of four AMRCFI evaluations.
//   k_cic_faces         the normal face averages n . <w> on the level's coarse-fine interface
//                       faces (Eq. cell2face along the face normal, from the two interior
//                       cells and the two CF ghost layers), corrected per connected component
//                       by one shift delta_c so that the interface and physical face sums of
//                       the component vanish (Eq. correctingFaceAvg).  One block per component;
//                       the sum is a fixed-order tree, so the result is deterministic.
#pragma once

namespace amr4 {

// The coarse data at the four times t_{-i} = t^{l-1} - i k (i = 0..3) and the two rows of
// I^(4)(k, eta) for them: row 0 the value weights, row 1 the weights of the time derivative.
struct CicTimes {
  const double* x[4];
  double w[2][4];
};

// Time combination of the coarse value at field offset o under both rows.
__device__ __forceinline__ void cic_pair(const CicTimes& ct, long long o, double& a, double& b) {
  const double v0 = ct.x[0][o], v1 = ct.x[1][o], v2 = ct.x[2][o], v3 = ct.x[3][o];
  a = ct.w[0][0] * v0 + ct.w[0][1] * v1 + ct.w[0][2] * v2 + ct.w[0][3] * v3;
  b = ct.w[1][0] * v0 + ct.w[1][1] * v1 + ct.w[1][2] * v2 + ct.w[1][3] * v3;
}

// By coarse parent (ratio 2): the 2^D children of one parent share its 5^D window; the x, y
// and z sums are folded dimension by dimension, for both time rows at once.
template <int D>
__global__ void k_cic_grp(const CfiGroup* __restrict__ list, long long n, const long long* __restrict__ side,
                          const PatchDesc* __restrict__ cpatches, CicTimes ct, double* __restrict__ out0,
                          double* __restrict__ out1) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CfiGroup& g = list[t];
  constexpr int NC = D == 3 ? 8 : 4;
  const int b0 = 2 * g.pos[0] * CFI_W, b1 = 2 * g.pos[1] * CFI_W, b2 = 2 * g.pos[2] * CFI_W;
  const long long src = g.src;
  PatchDesc cp{};
  if (src >= 0) cp = cpatches[g.cpatch];
  const long long* s = src >= 0 ? nullptr : side + (-1 - src) * (D == 3 ? 125 : 25);
  double acc[2][2][2][2];  // [row][x child][y child][z child]
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q >> 3][q & 1][(q >> 1) & 1][(q >> 2) & 1] = 0.0;
  for (int c2 = 0; c2 < (D == 3 ? CFI_W : 1); ++c2) {
    double by[2][2][2] = {};  // [row][x child][y child]
    for (int c1 = 0; c1 < CFI_W; ++c1) {
      double va[CFI_W], vb[CFI_W];
#pragma unroll
      for (int c0 = 0; c0 < CFI_W; ++c0) {
        const long long o = s == nullptr ? src + (long long)c1 * cp.sy + (long long)c2 * cp.sz + c0
                                         : s[(c2 * CFI_W + c1) * CFI_W + c0];
        cic_pair(ct, o, va[c0], vb[c0]);
      }
      double bx[2][2] = {};  // [row][x child]
#pragma unroll
      for (int c0 = 0; c0 < CFI_W; ++c0) {
        const double w0 = cfiw<double>(b0 + c0), w1 = cfiw<double>(b0 + CFI_W + c0);
        bx[0][0] += w0 * va[c0];
        bx[0][1] += w1 * va[c0];
        bx[1][0] += w0 * vb[c0];
        bx[1][1] += w1 * vb[c0];
      }
      const double wy0 = cfiw<double>(b1 + c1), wy1 = cfiw<double>(b1 + CFI_W + c1);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          by[r][a][0] += wy0 * bx[r][a];
          by[r][a][1] += wy1 * bx[r][a];
        }
    }
    const double wz0 = D == 3 ? cfiw<double>(b2 + c2) : 1.0, wz1 = D == 3 ? cfiw<double>(b2 + CFI_W + c2) : 0.0;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          acc[r][a][b][0] += wz0 * by[r][a][b];
          acc[r][a][b][1] += wz1 * by[r][a][b];
        }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (g.dst[c] >= 0) {
      out0[g.dst[c]] = acc[0][c & 1][(c >> 1) & 1][c >> 2];
      if (out1) out1[g.dst[c]] = acc[1][c & 1][(c >> 1) & 1][c >> 2];
    }
}

// One thread per CF ghost (any ratio): the full tensor-product window.
template <int D>
__global__ void k_cic(const CfiEntry* __restrict__ list, long long n, const long long* __restrict__ side,
                      const PatchDesc* __restrict__ cpatches, int r, CicTimes ct, double* __restrict__ out0,
                      double* __restrict__ out1) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CfiEntry e = list[t];
  const int b0 = (e.pos[0] * r + e.sub[0]) * CFI_W;
  const int b1 = (e.pos[1] * r + e.sub[1]) * CFI_W;
  const int b2 = (e.pos[2] * r + e.sub[2]) * CFI_W;
  PatchDesc cp{};
  if (e.src >= 0) cp = cpatches[e.cpatch];
  const long long* s = e.src >= 0 ? nullptr : side + (-1 - e.src) * (D == 3 ? 125 : 25);
  double a0 = 0.0, a1 = 0.0;
  for (int c2 = 0; c2 < (D == 3 ? CFI_W : 1); ++c2)
    for (int c1 = 0; c1 < CFI_W; ++c1) {
      const double wr = cfiw<double>(b1 + c1) * (D == 3 ? cfiw<double>(b2 + c2) : 1.0);
#pragma unroll
      for (int c0 = 0; c0 < CFI_W; ++c0) {
        const long long o = s == nullptr ? e.src + (long long)c1 * cp.sy + (long long)c2 * cp.sz + c0
                                         : s[(c2 * CFI_W + c1) * CFI_W + c0];
        double va, vb;
        cic_pair(ct, o, va, vb);
        const double w = cfiw<double>(b0 + c0) * wr;
        a0 += w * va;
        a1 += w * vb;
      }
    }
  out0[e.dst] = a0;
  if (out1) out1[e.dst] = a1;
}

constexpr int CIC_FACE_THREADS = 256;

// blockIdx.x = component c, its faces [cstart[c], cstart[c+1]).  phys (nullable): the sum of
// the component's physical face averages; delta (nullable) receives the shift.
__global__ void __launch_bounds__(CIC_FACE_THREADS)
k_cic_faces(const CicFace* __restrict__ faces, const int* __restrict__ cstart, Ptr3 w,
            const double* __restrict__ phys, double* __restrict__ out, double* __restrict__ delta) {
  pdl_wait();
  __shared__ double part[CIC_FACE_THREADS / 32];
  __shared__ double shift;
  const int c = blockIdx.x;
  const int i0 = cstart[c], i1 = cstart[c + 1];
  double acc = 0.0;
  for (int i = i0 + (int)threadIdx.x; i < i1; i += CIC_FACE_THREADS) {
    const CicFace f = faces[i];
    const double* x = f.dir == 0 ? w.p[0] : (f.dir == 1 ? w.p[1] : w.p[2]);  // no indexed parameter array
    // Eq. (cell2face) along the normal: 7/12 on the two cells next to the face, -1/12 on the
    // next ones; the interior cells are ghost - step and ghost - 2 step
    const double v = (7.0 * (x[f.ghost - f.step] + x[f.ghost]) - (x[f.ghost - 2 * f.step] + x[f.ghost + f.step])) *
                     (1.0 / 12.0);
    const double nv = f.side > 0 ? v : -v;
    out[i] = nv;
    acc += nv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CIC_FACE_THREADS / 32; ++k) s += part[k];
    const int nf = i1 - i0;
    const double d = nf > 0 ? -(s + (phys ? phys[c] : 0.0)) / (double)nf : 0.0;
    shift = d;
    if (delta) delta[c] = d;
  }
  __syncthreads();
  const double d = shift;
  for (int i = i0 + (int)threadIdx.x; i < i1; i += CIC_FACE_THREADS) out[i] += d;
}

}  // namespace amr4
