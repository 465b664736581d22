// Data migration after regridding (Sec. 5.4, last paragraph): the copy blocks between a new
// and an old hierarchy.  The AMRCFI part of the migration reuses k_cfi with entries whose
// windows lie in the new coarser level.
#pragma once

namespace amr4 {

// One row of CUDA blocks per copy block (blockIdx.y), a grid-stride loop over its cells.
// Every offset is checked against both fields' lengths; a violation is counted in *bad and
// the access skipped.
template <int D>
__global__ void k_migrate_copy(const MigrateBlock* __restrict__ blocks, const PatchDesc* __restrict__ npatches,
                               const PatchDesc* __restrict__ opatches, const double* __restrict__ xo, long long no,
                               double* __restrict__ xn, long long nn, unsigned* __restrict__ bad) {
  pdl_wait();
  const MigrateBlock b = blocks[blockIdx.y];
  const PatchDesc np = npatches[b.npatch], op = opatches[b.opatch];
  const long long ex = b.hi[0] - b.lo[0] + 1, ey = b.hi[1] - b.lo[1] + 1;
  const long long ez = D == 3 ? b.hi[2] - b.lo[2] + 1 : 1;
  const long long n = ex * ey * ez;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % ex), j = (int)((t / ex) % ey), k = (int)(t / (ex * ey));
    const int g0 = b.lo[0] + i, g1 = b.lo[1] + j, g2 = D == 3 ? b.lo[2] + k : 0;
    const long long dn = poff(np, g0 - np.lo[0], g1 - np.lo[1], D == 3 ? g2 - np.lo[2] : 0);
    const long long so = poff(op, g0 - op.lo[0], g1 - op.lo[1], D == 3 ? g2 - op.lo[2] : 0);
    if (dn < 0 || dn >= nn || so < 0 || so >= no) {
      atomicAdd(bad, 1u);
      continue;
    }
    xn[dn] = xo[so];
  }
}

}  // namespace amr4
