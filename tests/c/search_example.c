/* A search through the C ABI alone: create, iterate, read the coherence.
 * Exit status: 0 on success, 3 when the library reports TRSTMI_ECUDA (no
 * usable GPU), 1 on any other error. */
#include <stdio.h>

#include "trstmi.h"

int main(void) {
  trstmi_options o;
  trstmi_default_options(&o);
  o.K = 256;
  o.precision = TRSTMI_FP32;
  trstmi_handle h = NULL;
  int rc = trstmi_create(64, 8, 1, &o, &h);
  if (rc != TRSTMI_OK) {
    printf("trstmi_create: %s\n", trstmi_strerror(rc));
    return rc == TRSTMI_ECUDA ? 3 : 1;
  }
  trstmi_step_info info;
  double mu = 0.0, welch = 0.0;
  rc = trstmi_step(h, 100, &info);
  if (rc == TRSTMI_OK) rc = trstmi_coherence(h, &mu, &welch);
  printf("status %s, mu %.6f, Welch bound %.6f\n", trstmi_strerror(rc), mu, welch);
  trstmi_destroy(h);
  return rc == TRSTMI_OK ? 0 : 1;
}
