// Coarse-fine interface conditions of a subcycled level solve (Sec. 6.3, steps CIC-2 and
// CIC-3; Sec. 6.4, Eq. correctingFaceAvg).
//
//   k_cic_combine +     the CF ghost cells of level l at an intermediate time t*: AMRCFI of the
//   k_cic_grp3 (3-D),   level-(l-1) data at four equispaced coarse times, combined by the 2 x 4
//   k_cic_grp (2-D)     matrix I^(4)(k, eta) of Eq. (timeInterp) into the value at t* and its
//                       time derivative (ratio 2).  Both maps are linear, so the two time
//                       combinations of the coarse data are formed first and AMRCFI is applied
//                       to them: twice the AMRCFI arithmetic instead of four AMRCFI
//                       evaluations.  In 3-D the combinations are formed once per coarse window
//                       cell (k_cic_combine) -- the kernels are bound by GB300's FP64 rate, and
//                       a coarse cell lies in about 24 windows; k_cic_grp (2-D) forms them per
//                       window cell.
//   k_cic_faces_sum /   the normal face averages n . <w> on the level's coarse-fine interface
//   k_cic_faces_shift   faces (Eq. cell2face along the face normal, from the two interior
//                       cells and the two CF ghost layers), corrected per connected component
//                       by one shift delta_c so that the interface and physical face sums of
//                       the component vanish (Eq. correctingFaceAvg).  Two passes over chunks
//                       of each component's faces; every sum is a fixed-order tree, so the
//                       result is deterministic.
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

// The two time combinations of every coarse cell the level's AMRCFI windows read (3-D, ratio
// 2): each coarse value is combined once here instead of once per window that holds it
// (about 24 windows per cell on a box face).  y0 / y1 are indexed by field offset - base;
// y1 may be null (no derivative wanted).
__global__ void k_cic_combine(const long long* __restrict__ band, long long n, long long base, CicTimes ct,
                              double* __restrict__ y0, double* __restrict__ y1) {
  pdl_wait();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const long long o = band[t];
  double a, b;
  cic_pair(ct, o, a, b);
  y0[o - base] = a;
  if (y1) y1[o - base] = b;
}

// 3-D AMRCFI by coarse parent of the combined values, eight lanes per parent: lane c0 < 5
// takes the window cells of x offset c0 (the four parents of a warp, neighbours along the
// face, read adjacent rows) and folds its 25 cells through the y and z weights; the eight
// partial sums per lane go through shared memory, and lane j forms child j's x sum over the
// five lanes (value and derivative).  Every lane reaches the warp barrier.
constexpr int CIC_LANES = 8;
constexpr int CIC_GRP_THREADS = 128;

__global__ void __launch_bounds__(CIC_GRP_THREADS)
k_cic_grp3(const CfiGroup* __restrict__ list, long long n, const long long* __restrict__ side,
           const PatchDesc* __restrict__ cpatches, const double* __restrict__ y0, const double* __restrict__ y1,
           long long base, double* __restrict__ out0, double* __restrict__ out1) {
  pdl_wait();
  __shared__ double tsh[CIC_GRP_THREADS / CIC_LANES][CFI_W][8];  // [parent][c0][row*4 + 2 ychild + zchild]
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long t = tid / CIC_LANES;
  const int lane = (int)(threadIdx.x % CIC_LANES), gi = (int)(threadIdx.x / CIC_LANES);
  const bool live = t < n;
  const CfiGroup* g = live ? &list[t] : nullptr;
  if (live && lane < CFI_W) {
    const int c0 = lane;
    const int b1 = 2 * g->pos[1] * CFI_W, b2 = 2 * g->pos[2] * CFI_W;
    const long long src = g->src;
    long long sy = 0, sz = 0;
    if (src >= 0) {
      const PatchDesc& cp = cpatches[g->cpatch];
      sy = cp.sy;
      sz = cp.sz;
    }
    const long long* s = src >= 0 ? nullptr : side + (-1 - src) * 125;
    double tz[2][2][2] = {};  // [row][y child][z child]
    for (int c2 = 0; c2 < CFI_W; ++c2) {
      const double wz0 = cfiw<double>(b2 + c2), wz1 = cfiw<double>(b2 + CFI_W + c2);
      double ty[2][2] = {};  // [row][y child]
#pragma unroll
      for (int c1 = 0; c1 < CFI_W; ++c1) {
        const long long o = (s == nullptr ? src + (long long)c1 * sy + (long long)c2 * sz + c0
                                          : s[(c2 * CFI_W + c1) * CFI_W + c0]) - base;
        const double va = y0[o], vb = y1 ? y1[o] : 0.0;
        const double wy0 = cfiw<double>(b1 + c1), wy1 = cfiw<double>(b1 + CFI_W + c1);
        ty[0][0] += wy0 * va;
        ty[0][1] += wy1 * va;
        ty[1][0] += wy0 * vb;
        ty[1][1] += wy1 * vb;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          tz[r][b][0] += wz0 * ty[r][b];
          tz[r][b][1] += wz1 * ty[r][b];
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int z = 0; z < 2; ++z) tsh[gi][c0][r * 4 + 2 * b + z] = tz[r][b][z];
  }
  __syncwarp();
  if (!live) return;
  const long long dst = g->dst[lane];
  if (dst < 0) return;
  const int a = lane & 1, b = (lane >> 1) & 1, z = lane >> 2;  // child = x + 2 y + 4 z
  const int bx = (2 * g->pos[0] + a) * CFI_W;
  double v0 = 0.0, v1 = 0.0;
#pragma unroll
  for (int c0 = 0; c0 < CFI_W; ++c0) {
    const double wx = cfiw<double>(bx + c0);
    v0 += wx * tsh[gi][c0][2 * b + z];
    v1 += wx * tsh[gi][c0][4 + 2 * b + z];
  }
  out0[dst] = v0;
  if (out1) out1[dst] = v1;
}

constexpr int CIC_FACE_THREADS = 256;

// Fixed-order block sum: per-thread partials, a shuffle tree per warp, the eight warp partials
// in order.  Every thread of the block returns the total.
__device__ __forceinline__ double cic_block_sum(double acc, double* part) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __syncthreads();  // part may still be read from a previous use
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CIC_FACE_THREADS / 32; ++k) s += part[k];
  return s;
}

// Pass 1, one block per chunk of one component's faces: n . <w> of each face (Eq. cell2face
// along the normal: 7/12 on the two cells next to the face, -1/12 on the next ones; the
// interior cells are ghost - step and ghost - 2 step) into out, the chunk's sum into psum.
__global__ void __launch_bounds__(CIC_FACE_THREADS)
k_cic_faces_sum(const CicFace* __restrict__ faces, const CicChunk* __restrict__ chunks, Ptr3 w,
                double* __restrict__ out, double* __restrict__ psum) {
  pdl_wait();
  __shared__ double part[CIC_FACE_THREADS / 32];
  const CicChunk ch = chunks[blockIdx.x];
  double acc = 0.0;
  for (int i = ch.begin + (int)threadIdx.x; i < ch.end; i += CIC_FACE_THREADS) {
    const CicFace f = faces[i];
    const double* x = f.dir == 0 ? w.p[0] : (f.dir == 1 ? w.p[1] : w.p[2]);  // no indexed parameter array
    const double v = (7.0 * (x[f.ghost - f.step] + x[f.ghost]) - (x[f.ghost - 2 * f.step] + x[f.ghost + f.step])) *
                     (1.0 / 12.0);
    const double nv = f.side > 0 ? v : -v;
    out[i] = nv;
    acc += nv;
  }
  const double s = cic_block_sum(acc, part);
  if (threadIdx.x == 0) psum[blockIdx.x] = s;
}

// Pass 2, the same chunks: every block sums its component's chunk sums in chunk order (so all
// blocks of a component get the same bits), forms delta_c of Eq. (correctingFaceAvg) and
// adds it to its chunk; the component's first block stores delta_c.  phys (nullable): the
// sum of the component's physical face averages.
__global__ void __launch_bounds__(CIC_FACE_THREADS)
k_cic_faces_shift(const CicChunk* __restrict__ chunks, const int* __restrict__ ccstart,
                  const int* __restrict__ cstart, const double* __restrict__ psum,
                  const double* __restrict__ phys, double* __restrict__ out, double* __restrict__ delta) {
  pdl_wait();
  __shared__ double part[CIC_FACE_THREADS / 32];
  const CicChunk ch = chunks[blockIdx.x];
  const int c = ch.comp;
  double acc = 0.0;
  for (int k = ccstart[c] + (int)threadIdx.x; k < ccstart[c + 1]; k += CIC_FACE_THREADS) acc += psum[k];
  const double s = cic_block_sum(acc, part);
  const int nf = cstart[c + 1] - cstart[c];
  const double d = nf > 0 ? -(s + (phys ? phys[c] : 0.0)) / (double)nf : 0.0;
  if (threadIdx.x == 0 && (int)blockIdx.x == ccstart[c] && delta) delta[c] = d;
  for (int i = ch.begin + (int)threadIdx.x; i < ch.end; i += CIC_FACE_THREADS) out[i] += d;
}

// Face averages <x> (Eq. cell2face along the normal, no sign) on the interface faces
// [begin, end) of one single-box component, into the slots of its box problem's boundary
// data: the Dirichlet data w = w^I of the component's level problem.
__global__ void k_cic_face_bc(const CicFace* __restrict__ faces, const long long* __restrict__ slot, int begin,
                              int end, const double* __restrict__ x, double* __restrict__ out) {
  pdl_wait();
  const int i = begin + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= end) return;
  const CicFace f = faces[i];
  out[slot[i]] =
      (7.0 * (x[f.ghost - f.step] + x[f.ghost]) - (x[f.ghost - 2 * f.step] + x[f.ghost + f.step])) * (1.0 / 12.0);
}

}  // namespace amr4
