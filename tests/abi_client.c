/* A plain C99 caller of libetdm: include/etdm.h must compile as C (no C++ in
 * it) and every entry point must link.  Only calls that fail or answer before
 * any device work are made, so no GPU is needed; the program prints one line
 * per check and returns the number of failed checks. */
#include <pthread.h>
#include <stdio.h>
#include <string.h>

#include "etdm.h"

static int fails = 0;

/* a failing call without a handle on another thread */
static void *other_thread(void *arg) {
  etdm_handle *h = NULL;
  (void)arg;
  return etdm_init_basis(NULL, NULL, &h) == ETDM_ERR_INVALID_ARG ? (void *)1 : NULL;
}

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) ++fails;
}

int main(void) {
  etdm_options o;
  etdm_handle *h = (etdm_handle *)&o; /* any non-NULL value: must be reset */
  int64_t off = -1, len = -1;
  double g[4] = {0.0, 0.0, 0.0, 0.0};

  memset(&o, 0xff, sizeof(o));
  etdm_default_options(&o);
  check(o.precision == ETDM_PREC_FP64 && o.lbfgs_m == 3 && o.gamma == 0.25 &&
            o.beta0 == 1.0 && o.param == ETDM_PARAM_OCCVIRT && o.expm == ETDM_EXPM_EIG &&
            o.functional == ETDM_FUNC_KS && o.vgroup == 0,
        "default options");

  check(etdm_init_basis(NULL, &o, &h) == ETDM_ERR_INVALID_ARG && h == NULL,
        "init without a system fails and clears *out");
  check(strlen(etdm_last_error(NULL)) > 0, "the init failure has a message");
  check(etdm_init_batch(NULL, 0, &o, &h) == ETDM_ERR_INVALID_ARG && h == NULL,
        "an empty batch fails");

  check(etdm_num_systems(NULL) == 0, "no handle, no systems");
  check(etdm_system_layout(NULL, 0, &off, &len) == ETDM_ERR_INVALID_ARG, "layout needs a handle");
  check(etdm_system_handle(NULL, 0) == NULL, "no system handle without a handle");
  check(etdm_energy_grad(NULL, NULL, NULL, NULL, NULL) == ETDM_ERR_STATE, "energy_grad needs a handle");
  check(etdm_lbfgs_reset(NULL) == ETDM_ERR_STATE, "lbfgs_reset needs a handle");
  check(etdm_check(NULL, NULL) == ETDM_ERR_STATE, "check needs a handle");
  check(etdm_set_reference(NULL, 0, NULL, NULL) == ETDM_ERR_STATE, "set_reference needs a handle");
  check(etdm_array_bytes(NULL, ETDM_ARR_S) == -1, "no arrays without a handle");

  check(etdm_lbfgs_direction_noalloc(g, NULL, NULL, 17, 4, g, g, NULL) == ETDM_ERR_INVALID_ARG,
        "allocation-free direction: more pairs than its scratch holds");
  check(strstr(etdm_last_error(NULL), "scratch limit") != NULL, "... with the limit named");
  {
    pthread_t t;
    void *ok = NULL;
    check(pthread_create(&t, NULL, other_thread, NULL) == 0 && pthread_join(t, &ok) == 0 &&
              ok != NULL,
          "a failing init on another thread");
    check(strstr(etdm_last_error(NULL), "scratch limit") != NULL,
          "... leaves this thread's message as it was");
  }
  check(etdm_lbfgs_direction_noalloc(g, NULL, NULL, 0, 0, g, g, NULL) == ETDM_OK,
        "allocation-free direction: n = 0 returns at once");
  check(etdm_pair_gemm(NULL, NULL, NULL, 0, 0, 0, 0, 0, NULL) == ETDM_ERR_INVALID_ARG,
        "pair_gemm checks its sizes");

  etdm_free(NULL);
  check(1, "etdm_free(NULL) is a no-op");
  return fails;
}
