// Small-space buffers and entry of the OptDMD fit (Sec. 4.2); shared by the
// fit driver and the OptDMD kernels.
#pragma once

#include "common.cuh"

namespace dmd {

struct OptBufs {
  double *YD, *Phi, *RE, *G, *Ri, *H, *H2, *BC, *EtRE, *Gb, *Hh, *JtJt, *gt, *JtJ, *g, *Bk, *A, *p, *pt, *sd, *Z, *Wt,
      *Mlift;
  int* kinds;
  int32_t *si, *sinfo;
};

// Carves the buffers for T snapshots, rank r and sketch width l.
void carve_optdmd(Arena& a, int T, int r, int l, OptBufs& o);

// From the fit's B = Q^T X (l x T, ld l), U_B (l x l, leading r columns),
// T2 (Q = Q1 T2) and the exact-DMD model in `modal`: runs the fit and leaves
// the modes' small factor Mlift (l x r, Phi_R = Q1 Mlift) in o.Mlift; writes
// lambda and beta of `modal` (sigma is kept).
dmd_status optdmd_small(int T, int r, int l, const double* Bsnap, const double* UB, const double* T2, double* modal,
                        int32_t* info, double* stats, const dmd_optdmd_opts& opt, OptBufs& o, cudaStream_t st);

}  // namespace dmd
