/* A plain-C client of the library's C ABI (host-only calls, no GPU needed): creates a
 * two-level 2-D hierarchy, prints its field layout and the interface faces of level 1, then
 * regrids a tagged rectangle and prints the new boxes.  Used by tests/test_c_abi_client.py,
 * which compares the output with the Python binding's. */
#include <stdio.h>
#include <stdlib.h>

#include "amr4.h"

static int check(amr_status s, const char* where) {
  if (s != AMR_OK) {
    fprintf(stderr, "%s: status %d: %s\n", where, (int)s, amr_last_error());
    return 1;
  }
  return 0;
}

int main(void) {
  const int nboxes[2] = {1, 2};
  const int boxes[12] = {0, 0, 31, 31, /* level 1: */ 8, 8, 23, 27, 40, 36, 55, 51};
  amr_hierarchy_desc d;
  d.dim = 2;
  d.ratio = 2;
  d.n0[0] = 32;
  d.n0[1] = 32;
  d.n0[2] = 1;
  d.h0 = 1.0 / 32.0;
  d.nlevels = 2;
  d.nboxes = nboxes;
  d.boxes = boxes;
  amr_hierarchy* h = NULL;
  if (check(amr_hierarchy_create(&d, &h), "amr_hierarchy_create")) return 1;

  int npatch = 0;
  long long nelems = 0;
  if (check(amr_field_layout(h, &npatch, &nelems, NULL), "amr_field_layout")) return 1;
  amr_patch_info* info = (amr_patch_info*)malloc(sizeof(amr_patch_info) * (size_t)npatch);
  if (check(amr_field_layout(h, NULL, NULL, info), "amr_field_layout")) return 1;
  printf("layout %d %lld\n", npatch, nelems);
  for (int p = 0; p < npatch; ++p)
    printf("patch %d %d %lld %lld %lld\n", info[p].level, info[p].box, info[p].offset, info[p].stride_y,
           info[p].nelems);

  int nf = 0, nc = 0;
  if (check(amr_cic_faces(h, 1, &nf, &nc, NULL, NULL, NULL), "amr_cic_faces")) return 1;
  int* cell = (int*)malloc(sizeof(int) * 2 * (size_t)nf);
  int* face = (int*)malloc(sizeof(int) * (size_t)nf);
  int* comp = (int*)malloc(sizeof(int) * (size_t)nf);
  if (check(amr_cic_faces(h, 1, NULL, NULL, cell, face, comp), "amr_cic_faces")) return 1;
  long long sum = 0;
  for (int i = 0; i < nf; ++i) sum += (long long)(cell[2 * i] * 7 + cell[2 * i + 1] * 13 + face[i] * 3 + comp[i]);
  printf("faces %d %d %lld\n", nf, nc, sum);

  /* regrid: a tagged rectangle of level 0 */
  int tags[2 * 60];
  int nt = 0;
  for (int y = 10; y < 16; ++y)
    for (int x = 4; x < 14; ++x) {
      tags[2 * nt] = x;
      tags[2 * nt + 1] = y;
      ++nt;
    }
  const int ntags[1] = {nt};
  const int* tagp[1] = {tags};
  amr_regrid_params rp;
  rp.efficiency = 0.8;
  rp.min_width = 2;
  int new_nl = 0, nb[2] = {0, 0};
  if (check(amr_regrid(2, 2, d.n0, 2, ntags, tagp, &rp, &new_nl, nb, NULL, 0), "amr_regrid")) return 1;
  const int total = nb[0] + (new_nl > 1 ? nb[1] : 0);
  int* out = (int*)malloc(sizeof(int) * 4 * (size_t)total);
  if (check(amr_regrid(2, 2, d.n0, 2, ntags, tagp, &rp, &new_nl, nb, out, total), "amr_regrid")) return 1;
  printf("regrid %d", new_nl);
  for (int i = 0; i < 4 * total; ++i) printf(" %d", out[i]);
  printf("\n");

  free(out);
  free(cell);
  free(face);
  free(comp);
  free(info);
  amr_hierarchy_destroy(h);
  return 0;
}
