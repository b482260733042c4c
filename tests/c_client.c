/* A plain C99 client of include/momenti.h: the header compiles as C and the
 * library links and answers from C.  Uses only calls that need no device:
 * parameters and handle life cycle, argument errors, and the search's host
 * arithmetic.  Prints one line per check; exits non-zero on the first
 * failure. */
#include <math.h>
#include <stdio.h>

#include "momenti.h"

static int check(int ok, const char* what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  return ok ? 0 : 1;
}

int main(void) {
  momenti_params p;
  momenti_handle* h = NULL;
  int64_t idx[2] = {-1, -1};
  int32_t n = -1;
  const float dd[3] = {2.0f, 1.0f, 3.0f};
  const int64_t a[3] = {0, 100, 400};
  const int64_t b[3] = {50, 200, 500};
  double pr, fb;

  if (check(momenti_default_params(&p) == MOMENTI_OK && p.K == 8 && p.L == 200, "default params"))
    return 1;
  p.w = 10;
  if (check(momenti_create(&h, &p) == MOMENTI_OK && h != NULL, "create")) return 1;
  if (check(momenti_hash_all(h, NULL, MOMENTI_F32, 100, 1, 100, 0, NULL) == MOMENTI_ERR_ARG,
            "hash_all rejects a NULL series"))
    return 1;
  if (check(momenti_last_error(h) != NULL && momenti_last_error(h)[0] != '\0', "last_error"))
    return 1;
  momenti_destroy(h);
  momenti_destroy(NULL);

  pr = momenti_collision_probability(1.0, 4.0);
  if (check(pr > 0.0 && pr < 1.0, "collision probability in (0, 1)")) return 1;
  if (check(momenti_collision_probability(0.0, 4.0) == 1.0, "collision probability at R = 0"))
    return 1;
  fb = momenti_failure_bound(1.0, 8, 10, 8, 200, 2, 4.0);
  if (check(fb > 0.0 && fb < 1.0, "failure bound in (0, 1)")) return 1;
  if (check(isnan(momenti_failure_bound(1.0, 9, 10, 8, 200, 2, 4.0)), "failure bound i > K"))
    return 1;
  if (check(momenti_top_select(dd, a, b, 3, 2, 10, 1, idx, &n) == MOMENTI_OK && n == 2 &&
                idx[0] == 1 && idx[1] == 0,
            "top_select"))
    return 1;
  return 0;
}
