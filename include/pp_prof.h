/*
 * pp_prof.h -- diagnostics of libpp used by the benchmark: per-kernel-class
 * CUDA-event timing on the launching stream, and an FP64 FMA throughput probe.
 * None of these calls is part of the method; they allocate only CUDA events.
 */
#ifndef PP_PROF_H
#define PP_PROF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* kernel classes */
#define PP_K_NONE 0
#define PP_K_JACOBIAN 1      /* element block Jacobian (dual-number quadrature) */
#define PP_K_RESIDUAL 2      /* residual r(u, mu, t) */
#define PP_K_STAGE_MATVEC 3  /* alpha M x + beta J x / J^T x over the block-sparse Jacobian */
#define PP_K_BLOCK_APPLY 4   /* block-Jacobi inverse application (normal / transposed) */
#define PP_K_BLOCK_INVERSE 5 /* batched Gauss-Jordan inversion of the stage diagonal blocks */
#define PP_K_KRYLOV 6        /* fused multi-dot / update / norm reductions */
#define PP_K_OTHER 7         /* vector combinations, QoI and column-sum kernels */
#define PP_K_STAGE_MATVEC32 8  /* FP32 block-sparse product (mixed-precision inner solves) */
#define PP_K_BLOCK_APPLY32 9   /* FP32 block-Jacobi application */
#define PP_K_KRYLOV32 10       /* FP32 Krylov reductions */
#define PP_K_STAGE_OP 11       /* FP64 stage operator with the preconditioner folded in, x + B x */
#define PP_K_FOLD 12           /* products B = -c J_off D^-1 forming that operator (FP64 or FP32) */
#define PP_K_STAGE_OP32 13     /* FP32 folded stage operator of the mixed-precision inner solves */
#define PP_K_COUNT 14

/* Starts timing every launch of kernel class `kind` (one class at a time; PP_K_NONE
   stops).  Resets the accumulated totals.  Not thread-safe: one host thread drives libpp. */
int pp_prof_select(int kind);
/* Synchronizes the device and returns, for the selected class since pp_prof_select,
   the number of launches and the summed event time in milliseconds. */
int pp_prof_read(int64_t* launches, double* total_ms);
/* Counts launches of every class since the last pp_prof_select (no events). */
int pp_prof_counts(int64_t* counts /* [PP_K_COUNT] */);

/* Iteration counts of the last sweeps on ctx: stage Newton iterations and GMRES
   iterations of the last primal sweep; GMRES iterations of the last tangent and of
   the last adjoint sweep.  Any pointer may be NULL. */
struct pp_ctx;
int pp_sweep_counts(const struct pp_ctx* ctx, int64_t* newton, int64_t* gmres_primal, int64_t* gmres_tangent,
                    int64_t* gmres_adjoint);

/* Applies one operator of the stored linearization of DIRK step `step` (0 .. Nt-1), stage
   `stage` (0 .. 2) to x, for tests of the stored blocks against dense products of the same
   matrices (c = a_ii dt, D = block diagonal of M - c J; the operators of Eqs.
   dirk-sens-mvp and uns-disc-adj-dirk2):
     kind 0: y = (M - c J) x                       trans 1: y = (M - c J)^T x
     kind 1: y = D^{-1} x (block-Jacobi inverse)   trans 1: y = D^{-T} x
     kind 2: y = (M - c J) D^{-1} x (the folded operator I + B)
                                                   trans 1: y = (M - c J)^T D^{-T} x
   prec 0 uses the FP64 data, prec 1 the FP32 copies of PP_PREC_MIXED (x, y cast through
   FP32).  x, y: DEVICE FP64 [N_u], distinct.  With a checkpointed linearization the
   step's segment is recomputed first.  Errors: PP_ESTATE (no sweep stored, or the
   requested data is not stored in this mode), PP_EINVAL. */
int pp_stage_apply(struct pp_ctx* ctx, int step, int stage, int kind, int trans, int prec, const double* x,
                   double* y);

/* Measures the device's FP64 FMA throughput (TFLOP/s, 2 flops per FMA) with an
   unrolled dependent-chain kernel over all SMs; returns PP_OK or PP_ECUDA. */
int pp_measure_fp64_peak(int device, double* tflops);

#ifdef __cplusplus
}
#endif
#endif
