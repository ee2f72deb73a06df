/* A C program on the C ABI of libsu3 alone (no Python): the calls that need
 * no GPU -- version, argument checks, the host-side decomposition planner.
 * Built and run by tests/test_abi.py. */
#include <stdio.h>
#include <string.h>

#include "su3.h"

int main(void) {
  su3_handle h = NULL;
  int nsub = 0;
  long long halo = 0;
  if (strncmp(su3_version(), "libsu3", 6) != 0) return 1;
  /* odd extent: rejected before any device work */
  if (su3_create(4, 4, 4, 5, 5.7, 1, SU3_COLD, &h) != SU3_EINVAL || h != NULL) return 2;
  if (strstr(su3_last_error(), "extent") == NULL) return 3;
  if (su3_destroy(NULL) != SU3_OK) return 4;
  /* the paper's np = 16 row of the 32^4 column, planned on the host */
  if (su3_decomp_plan(32, 32, 32, 32, 4, 2, 1, &nsub, &halo) != SU3_OK) return 5;
  if (nsub != 16) return 6;
  /* ghost cells per 16^4 sublattice: 8 faces of 16^3 and 12 edges of 16^2 */
  if (halo != 4LL * 16 * (8LL * 4096 + 12LL * 256)) return 7;
  if (su3_decomp_plan(32, 32, 32, 32, 4, 3, 1, &nsub, &halo) != SU3_EINVAL) return 8;
  printf("c abi ok: %s, np %d, halo links per sweep %lld\n", su3_version(), nsub, halo);
  return 0;
}
