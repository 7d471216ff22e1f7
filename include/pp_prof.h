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
#define PP_K_ARNOLDI 14        /* the Gram-Schmidt passes of one FP64 Arnoldi step (3 launches) */
#define PP_K_ARNOLDI32 15      /* the same in FP32 (mixed-precision inner solves) */
#define PP_K_COUNT 16

/* Starts timing every launch of kernel class `kind` (PP_K_NONE stops), and only that class.
   Resets the accumulated totals of every class.  Not thread-safe: one host thread drives
   libpp.  At most 262144 launches of a class are timed. */
int pp_prof_select(int kind);
/* Times one launch in `stride` of each timed class (default 1: every launch), so that the
   events disturb the timed work less; classes that count bytes per group of launches (the
   Arnoldi steps) are sampled by whole groups.  Applies from the next pp_prof_select. */
int pp_prof_sample(int stride);
/* Adds class `kind` to the timed classes without resetting the totals. */
int pp_prof_also(int kind);
/* Synchronizes the device and returns, for the class given to pp_prof_select, the number
   of timed launches and their summed event time in milliseconds. */
int pp_prof_read(int64_t* launches, double* total_ms);
/* As pp_prof_read for any timed class, plus the algorithmic bytes of the timed launches
   where the class counts them (PP_K_ARNOLDI*: (2k + 3) n words per Arnoldi step against k
   basis vectors of length n: one classical Gram-Schmidt pass reads V and w for the
   projections, then V and w again and writes w for the update and norm); 0 otherwise. */
int pp_prof_read_class(int kind, int64_t* launches, double* total_ms, double* bytes);
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

/* All eigenvalues of an n x n upper Hessenberg matrix H (HOST, row-major, leading dimension
   ld >= n; overwritten) by the Francis double-shift QR iteration used by pp_floquet; host
   code only (no GPU needed).  wr, wi: HOST [n].  Returns PP_OK, PP_EINVAL or PP_ENOCONV. */
int pp_hessenberg_eigvals(int n, double* H, int ld, double* wr, double* wi);

/* Measures the device's FP64 FMA throughput (TFLOP/s, 2 flops per FMA): 16 independent FMA
   chains per thread, 2048 threads per SM, about 0.2 s per run, best of 5 runs.  sm_mhz
   (nullable) receives the SM clock of the best run, measured inside the kernel from the SM
   cycle counter against the global timer.  Returns PP_OK or PP_ECUDA. */
int pp_measure_fp64_peak(int device, double* tflops);
int pp_measure_fp64_peak_clock(int device, double* tflops, double* sm_mhz);

#ifdef __cplusplus
}
#endif
#endif
