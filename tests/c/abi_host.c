/* A plain C99 client of include/odmd.h: the header compiles as strict C, the library links
 * and its host-side entry points (configuration, workspace size, argument checks, error
 * strings) answer without a GPU.  Prints "ok" and exits 0, or names the first failure. */
#include <stdio.h>
#include <string.h>

#include "odmd.h"

#define EXPECT(cond)                                               \
  do {                                                             \
    if (!(cond)) {                                                 \
      fprintf(stderr, "abi_host: failed %s (line %d)\n", #cond, __LINE__); \
      return 1;                                                    \
    }                                                              \
  } while (0)

int main(void) {
  odmd_config cfg;
  size_t bytes = 0, small = 0;
  double s[4];
  int32_t r = -1;
  const char* msg;

  EXPECT(odmd_config_default(&cfg, 393216, 40) == ODMD_OK);
  EXPECT(cfg.n == 393216 && cfg.r_max == 40 && cfg.prec == ODMD_FP64 && cfg.flags == 0u);
  EXPECT(odmd_footprint(&cfg, &bytes) == ODMD_OK);
  /* two float planes of N x (r_max + slack) columns at least */
  EXPECT(bytes > (size_t)2 * 393216 * (size_t)(cfg.r_max + cfg.slack) * 4);

  EXPECT(odmd_config_default(&cfg, 1000, 8) == ODMD_OK);
  EXPECT(odmd_footprint(&cfg, &small) == ODMD_OK);
  EXPECT(small > 0 && small < bytes);

  /* out-of-range configurations are refused with the reason */
  EXPECT(odmd_config_default(&cfg, 1000, 65) == ODMD_OK);
  EXPECT(odmd_footprint(&cfg, &small) == ODMD_ERR_ARG);
  msg = odmd_last_error(NULL);
  EXPECT(msg != NULL && strstr(msg, "r_max") != NULL);
  EXPECT(odmd_config_default(&cfg, 0, 8) == ODMD_OK && cfg.n == 0);  /* filled, checked later */
  EXPECT(odmd_footprint(&cfg, &small) == ODMD_ERR_ARG);
  EXPECT(odmd_config_default(NULL, 10, 8) == ODMD_ERR_ARG);
  EXPECT(odmd_config_default(&cfg, 1000, 8) == ODMD_OK);
  cfg.flags = ODMD_CUDA_CORES | ODMD_NO_PIPELINE;
  EXPECT(odmd_footprint(&cfg, &small) == ODMD_OK);       /* the two defined flags */
  cfg.flags = 4u;
  EXPECT(odmd_footprint(&cfg, &small) == ODMD_ERR_ARG);  /* unknown bits */
  EXPECT(odmd_footprint(NULL, &small) == ODMD_ERR_ARG);

  /* every limit the header states is enforced */
  {
    odmd_config c;
    EXPECT(odmd_config_default(&c, 2147483648LL, 8) == ODMD_OK);
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* n above 2^31 - 1 */
    EXPECT(odmd_config_default(&c, 1000, 0) == ODMD_OK);
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* r_max below 1 */
    EXPECT(odmd_config_default(&c, 1000, 64) == ODMD_OK);
    EXPECT(odmd_footprint(&c, &small) == ODMD_OK);      /* r_max 64 is the top */
    c.slack = 33;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* slack above 32 */
    c.slack = -1;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG);
    c.slack = 32;
    EXPECT(odmd_footprint(&c, &small) == ODMD_OK);
    c.trunc_tol = 1e-14;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* tau below 1e-13 */
    c.trunc_tol = 1.0;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* tau not below 1 */
    c.trunc_tol = 1e-10;
    c.prec = (odmd_precision)3;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* no such precision */
    c.prec = ODMD_BF16;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG); /* refused, with the reason */
    c.prec = ODMD_FP32;
    c.refine_every = -1;
    EXPECT(odmd_footprint(&c, &small) == ODMD_ERR_ARG);
    c.refine_every = 10;
    EXPECT(odmd_footprint(&c, &small) == ODMD_OK);
  }

  /* the allocation-free check refuses bad arguments before it touches the device (the
   * pointers below are never dereferenced: each call fails its argument checks first) */
  {
    const double* fake = (const double*)(uintptr_t)256;
    double err = 0.0;
    int32_t pass = 0;
    EXPECT(odmd_check_noalloc(NULL, fake, 10, 1e-5, NULL, &err, &pass) == ODMD_ERR_ARG);
    EXPECT(odmd_check_noalloc(fake, fake, 0, 1e-5, NULL, &err, &pass) == ODMD_ERR_ARG);
    EXPECT(odmd_check_noalloc(fake, fake, 33554433, 1e-5, NULL, &err, &pass) == ODMD_ERR_ARG);
    msg = odmd_last_error(NULL);
    EXPECT(msg != NULL && strstr(msg, "33554432") != NULL);
  }

  /* every handle call refuses a NULL handle before it touches the device */
  EXPECT(odmd_update(NULL, NULL) == ODMD_ERR_ARG);
  EXPECT(odmd_predict(NULL, NULL, 0, NULL, 0) == ODMD_ERR_ARG);
  EXPECT(odmd_get_rank(NULL, &r) == ODMD_ERR_ARG);
  EXPECT(odmd_get_singular_values(NULL, s, 4, &r) == ODMD_ERR_ARG);
  EXPECT(odmd_checkpoint_size(NULL, &small) == ODMD_ERR_ARG);
  EXPECT(odmd_destroy(NULL) == ODMD_ERR_ARG);
  msg = odmd_last_error(NULL);
  EXPECT(msg != NULL && strstr(msg, "NULL") != NULL);

  printf("ok\n");
  return 0;
}
