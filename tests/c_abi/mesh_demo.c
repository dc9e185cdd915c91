/* A plain C consumer of the library's C ABI (include/gbs_mpo.h): builds the lossy
 * squeezed initial MPO, applies a beam-splitter mesh read from a text file, and
 * prints the trace, the per-mode photon numbers, the largest operator entanglement,
 * the summed discarded weight, a checkpoint round trip and one App. C estimate.
 *
 * Usage: mesh_demo <mesh.txt>
 *   mesh.txt: "M d chi r eta n_gates" on the first line, then one "k theta phi" line
 *   per gate, then M final phases on one line.
 * Exit code 0 on success, the mpo_status of the first failing call otherwise. */
#include <stdio.h>
#include <stdlib.h>

#include "gbs_mpo.h"

#define CHECK(call)                                                              \
  do {                                                                           \
    mpo_status s_ = (call);                                                      \
    if (s_ != MPO_OK) {                                                          \
      fprintf(stderr, "%s failed: %s\n", #call, mpo_status_string(s_));          \
      return (int)s_;                                                            \
    }                                                                            \
  } while (0)

int main(int argc, char** argv) {
  if (argc < 2) { fprintf(stderr, "usage: %s mesh.txt\n", argv[0]); return 1; }
  FILE* f = fopen(argv[1], "r");
  if (!f) { perror("fopen"); return 1; }
  int M, d, chi, ng;
  double r, eta;
  if (fscanf(f, "%d %d %d %lf %lf %d", &M, &d, &chi, &r, &eta, &ng) != 6) { fclose(f); return 1; }
  int* k = malloc(sizeof(int) * ng);
  double* th = malloc(sizeof(double) * ng);
  double* ph = malloc(sizeof(double) * ng);
  double* fp = malloc(sizeof(double) * M);
  double* rr = malloc(sizeof(double) * M);
  double* ee = malloc(sizeof(double) * M);
  for (int i = 0; i < ng; ++i)
    if (fscanf(f, "%d %lf %lf", &k[i], &th[i], &ph[i]) != 3) { fclose(f); return 1; }
  for (int j = 0; j < M; ++j)
    if (fscanf(f, "%lf", &fp[j]) != 1) { fclose(f); return 1; }
  fclose(f);
  for (int j = 0; j < M; ++j) { rr[j] = r; ee[j] = eta; }

  mpo_params p = {0};
  p.M = M; p.d = d; p.n_cap = 0; p.batch = 1; p.prec = MPO_FP64; p.chi_max = &chi; p.cuda_stream = NULL;
  mpo_handle h = NULL;
  CHECK(mpo_init_lossy_squeezed(&h, &p, rr, ee));

  double* disc = malloc(sizeof(double) * ng);
  CHECK(mpo_sweep_mesh(h, &ng, k, th, ph, fp, disc));
  double tr = 0.0, dsum = 0.0;
  double* n1 = malloc(sizeof(double) * M);
  double* n2 = malloc(sizeof(double) * M);
  CHECK(mpo_observables(h, &tr, n1, n2, 1));
  double* S = malloc(sizeof(double) * (M + 1));
  double smax = 0.0;
  CHECK(mpo_operator_entropy(h, S, NULL, &smax));
  for (int i = 0; i < ng; ++i) dsum += disc[i];

  /* checkpoint round trip: save, reset, load, the trace comes back */
  size_t bytes = 0;
  CHECK(mpo_checkpoint_bytes(h, &bytes));
  void* ck = malloc(bytes);
  CHECK(mpo_save(h, ck, bytes, ng));
  CHECK(mpo_reset(h));
  long long cursor = -1;
  CHECK(mpo_load(h, ck, bytes, &cursor));
  double tr2 = 0.0;
  CHECK(mpo_observables(h, &tr2, NULL, NULL, 1));

  /* one App. C point: r = 0.88, mu = 0.3, theta = pi/4, n_max = 8 */
  double ar = 0.88, amu = 0.3, ath = 0.78539816339744831, aS = 0.0;
  CHECK(mpo_asymptotic_ee(1, 8, &ar, &amu, &ath, 1.0, &aS, NULL, NULL, 0));

  printf("trace %.17g\n", tr);
  printf("n_mean");
  for (int j = 0; j < M; ++j) printf(" %.17g", n1[j]);
  printf("\nS_max %.17g\ndiscarded_sum %.17g\n", smax, dsum);
  printf("checkpoint cursor %lld trace %.17g\n", cursor, tr2);
  printf("asymptotic_S1 %.17g\n", aS);
  mpo_destroy(h);
  free(k); free(th); free(ph); free(fp); free(rr); free(ee); free(disc); free(n1); free(n2); free(S); free(ck);
  return 0;
}
