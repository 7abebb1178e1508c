/* A plain C client of the library: uses only include/isam.h, libisam and the
 * CUDA runtime.  Reads a geometry and an image, applies A and A^H on the
 * device, writes s = A eta and A^H s.
 *
 *   isam_c_client nx nk nz k_min k_max dx na z0 a1 a2 a3 a4 eta.bin s.bin aHs.bin
 *
 * eta.bin: nx*nz complex64 (interleaved float re, im); s.bin: nx*nk float;
 * aHs.bin: nx*nz complex64.  Exit status 0 on success. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "isam.h"

static int fail(const char* what, int st) {
  fprintf(stderr, "%s failed: %d\n", what, st);
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 16) {
    fprintf(stderr, "usage: %s nx nk nz k_min k_max dx na z0 a1 a2 a3 a4 eta s aHs\n", argv[0]);
    return 2;
  }
  isam_params p = {0};
  p.nx = atoi(argv[1]);
  p.ny = 1;
  p.nk = atoi(argv[2]);
  p.nz = atoi(argv[3]);
  p.k_min = atof(argv[4]);
  p.k_max = atof(argv[5]);
  p.dx = atof(argv[6]);
  p.na = atof(argv[7]);
  p.z0 = atof(argv[8]);
  p.n_disp = 4;
  for (int i = 0; i < 4; ++i) p.disp[i] = atof(argv[9 + i]);
  p.precision = ISAM_FP32;
  const size_t n_img = (size_t)p.nx * p.nz, n_spec = (size_t)p.nx * p.nk;

  float* h_eta = (float*)malloc(2 * n_img * sizeof(float));
  float* h_s = (float*)malloc(n_spec * sizeof(float));
  float* h_a = (float*)malloc(2 * n_img * sizeof(float));
  FILE* f = fopen(argv[13], "rb");
  if (!f || fread(h_eta, sizeof(float), 2 * n_img, f) != 2 * n_img) return fail("read eta", 0);
  fclose(f);

  void *d_eta = NULL, *d_s = NULL, *d_a = NULL;
  if (cudaMalloc(&d_eta, 2 * n_img * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&d_s, n_spec * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&d_a, 2 * n_img * sizeof(float)) != cudaSuccess)
    return fail("cudaMalloc", 0);
  cudaMemcpy(d_eta, h_eta, 2 * n_img * sizeof(float), cudaMemcpyHostToDevice);

  isam_plan* plan = NULL;
  isam_status st = isam_plan_create(&p, NULL, &plan);
  if (st != ISAM_OK) return fail(isam_status_string(st), st);
  if ((st = isam_forward(plan, d_eta, d_s)) != ISAM_OK) return fail("isam_forward", st);
  if ((st = isam_adjoint(plan, d_s, d_a)) != ISAM_OK) return fail("isam_adjoint", st);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail("cudaDeviceSynchronize", 0);
  cudaMemcpy(h_s, d_s, n_spec * sizeof(float), cudaMemcpyDeviceToHost);
  cudaMemcpy(h_a, d_a, 2 * n_img * sizeof(float), cudaMemcpyDeviceToHost);
  isam_plan_destroy(plan);

  f = fopen(argv[14], "wb");
  fwrite(h_s, sizeof(float), n_spec, f);
  fclose(f);
  f = fopen(argv[15], "wb");
  fwrite(h_a, sizeof(float), 2 * n_img, f);
  fclose(f);
  cudaFree(d_eta);
  cudaFree(d_s);
  cudaFree(d_a);
  free(h_eta);
  free(h_s);
  free(h_a);
  return 0;
}
