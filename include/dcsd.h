/*
 * dcsd.h -- C ABI of the GB300 two-determinant CCSD / DCSD residual engine.
 *
 * The method is 2D-CCSD and its distinguishable-cluster variant 2D-DCSD of
 * Schraivogel & Kats, "Two Determinant Distinguishable Cluster" (arXiv
 * 2401.11935), Section II, Eqs. 2-4: the singles/doubles amplitude residuals
 * of an open-shell singlet or M_s = 0 triplet built on the two determinants
 * Phi_A (core^2, t alpha, u beta) and Phi_B (core^2, u alpha, t beta) of
 * Fig. 1, with the coupling W and the 2x2 effective Hamiltonian whose
 * eigenvalues are the singlet (dE_A + W) and triplet (dE_A - W) energies.
 *
 * Conventions shared by every call
 * --------------------------------
 * Spatial orbitals (n = n_c + 2 + n_v): core 0..n_c-1, t = n_c, u = n_c+1,
 * external virtuals n_c+2..n-1.  Two-electron integrals are density fitted:
 * (pq|rs) = sum_L B[L][p][q] B[L][r][s], B symmetric in (p,q).
 *
 * Amplitudes and residuals are normal-ordered to Phi_A (ref = 0) or Phi_B
 * (ref = 1).  With o = n_c + 1 and v = n_v + 1 per spin, the per-spin index
 * lists are
 *     ref 0: alpha occ (core..., t)  beta occ (core..., u)
 *            alpha vir (u, V...)     beta vir (t, V...)
 *     ref 1: alpha occ (core..., u)  beta occ (core..., t)
 *            alpha vir (t, V...)     beta vir (u, V...)
 * and the arrays are row-major doubles
 *     T1a, T1b  [o][v]
 *     T2aa, T2bb [o][o][v][v]   antisymmetric in (i,j) and in (a,b)
 *     T2ab      [o][o][v][v]    (alpha occ i, beta occ j, alpha vir a, beta vir b).
 * The excitation Phi_ref -> the other determinant is T2ab[o-1][o-1][0][0]
 * in both frames.  It is not a free amplitude, and the library sets it
 * whatever the array holds (and returns that value in solved amplitudes):
 * for the 2D methods by the C-condition <other|exp(T)|ref> = 0 of the
 * two-determinant wave operator, i.e. to -T1a[o-1][0] * T1b[o-1][0] (the
 * internal singles t alpha -> u alpha and u beta -> t beta of frame A, their
 * flips in frame B), which is zero in the CAS case (t and u in different
 * irreps, Section II, text after Eq. 4) and not in the IAS case (same
 * irrep); for the fixed-reference methods to the fixed value (+1 or -1).
 * Its gradient in dcsd_vjp is zero; the derivative flows to the singles.
 * Fock matrices passed to dcsd_init are those of Phi_A; for ref = 1 the
 * library uses the alpha matrix as beta and vice versa (spin flip).
 *
 * Ownership and errors: every function returns a dcsd_status; no exception
 * or abort crosses the ABI.  A context owns all device memory it allocates
 * (freed by dcsd_destroy).  Pointers passed to a call are borrowed for the
 * duration of that call only.  Device pointers must stay valid until the
 * work enqueued on the context's stream has finished.  dcsd_last_error
 * returns a message owned by the context, valid until the next call.
 */
#ifndef DCSD_H
#define DCSD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DCSD_OK = 0,
    DCSD_ERR_INVALID_ARG = 1,  /* bad pointer, size, enum value or layout  */
    DCSD_ERR_OOM = 2,          /* device allocation failed                 */
    DCSD_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed        */
    DCSD_ERR_NOT_CONVERGED = 4,/* dcsd_solve hit maxiter                   */
    DCSD_ERR_TIMEOUT = 5,      /* a bounded device wait gave up            */
    DCSD_ERR_NUMERIC = 6,      /* NaN/Inf in a residual or energy          */
    DCSD_ERR_NO_DEVICE = 7     /* no CUDA device of compute capability 10.3 */
} dcsd_status;

/* Methods.  0, 1: the two-determinant 2D-CCSD / 2D-DCSD of Section II
 * (Eqs. 2-4).  2..5: the fixed-reference FR-CCSD / FR-DCSD of the paper's
 * introduction (Section I): the doubles amplitude of the excitation
 * Phi_ref -> other determinant is held at a fixed value, +1 for the
 * open-shell singlet (_S) or -1 for the M_s = 0 triplet (_T) in this
 * library's phase of Phi_B (Phi_B = E_{A->B} Phi_A, singlet Phi_A + Phi_B),
 * all other amplitudes obey the single-reference CCSD / DCSD equations on
 * Phi_ref, and there are no M W terms.  The FR energy is the single-reference
 * Delta E = <ref|H_N exp(T)|ref>, which includes the fixed amplitude. */
typedef enum {
    DCSD_CCSD = 0,
    DCSD_DCSD = 1,
    DCSD_FR_CCSD_S = 2,
    DCSD_FR_DCSD_S = 3,
    DCSD_FR_CCSD_T = 4,
    DCSD_FR_DCSD_T = 5
} dcsd_method;
typedef enum { DCSD_MEM_HOST = 0, DCSD_MEM_DEVICE = 1 } dcsd_mem_kind;

/* Arithmetic of the dense contractions (ladder, ring, DF builds).  The
 * orbital-energy denominators, DIIS, energies, residual norm and the 2x2
 * effective Hamiltonian are always FP64. */
typedef enum {
    DCSD_PREC_FP64 = 0,   /* FP64 on CUDA cores                              */
    DCSD_PREC_BF16 = 1,   /* BF16 operands on tcgen05 tensor cores, FP32 acc */
    DCSD_PREC_BF16X3 = 2, /* split operands hi+mid, 3 BF16 products          */
    DCSD_PREC_MIXED = 3,  /* dcsd_solve only: BF16, BF16X6, FP64 (see below) */
    DCSD_PREC_BF16X6 = 4  /* split hi+mid+lo, 6 BF16 products (FP32-class)  */
} dcsd_precision;

typedef struct dcsd_ctx dcsd_ctx;

typedef struct {
    int n_c;   /* doubly occupied (correlated) spatial orbitals, >= 0 */
    int n_v;   /* external virtual spatial orbitals, >= 1            */
    int naux;  /* density-fitting functions, >= 1                    */
} dcsd_dims;

typedef struct {
    int method;         /* dcsd_method                                      */
    int ref;            /* 0 = Phi_A, 1 = Phi_B                             */
    int precision;      /* dcsd_precision                                   */
    int maxiter;        /* iteration cap (e.g. 100)                         */
    int diis_n;         /* DIIS history length, 0..16 (0 = Jacobi only)     */
    double tol;         /* convergence: max |R| <= tol                      */
    double switch_tol;  /* MIXED: switch BF16 -> BF16X6 when max|R| < this, or
                           when max|R| has not halved in 6 iterations      */
    int use_guess;      /* 1: start from the T passed in, 0: from T = 0      */
    double polish_tol;  /* MIXED: leave plain BF16X6 when max|R| < this, or
                           when max|R| has not halved in 4 BF16X6 iterations,
                           for defect correction: an outer step evaluates the
                           FP64 residual R64(T) and e = R_X6(T) - R64(T) at
                           the same T, inner BF16X6 steps iterate on
                           R_X6 - e; convergence (max|R64| <= tol) is tested
                           on outer steps only.  0 keeps plain BF16X6 to the
                           end.  The tensor cores accumulate in FP32, whose
                           rounding error in long contractions limits the
                           energies of a plain BF16X6 solve; with defect
                           correction the converged T solves the FP64
                           equations */
} dcsd_solve_opts;

typedef struct {
    double dEA;       /* Delta E_A = <A|H_N exp(T_A)|A>  (Eq. 2)            */
    double W;         /* <B|H_N exp(T_A)|A>, coupling of the two references */
    double E_S;       /* singlet correlation energy dE_A + W (FR methods:
                         dE_A for the _S methods, NaN for the _T ones)     */
    double E_T;       /* triplet correlation energy dE_A - W (FR methods:
                         dE_A for the _T methods, NaN for the _S ones)     */
    double max_r;     /* max |R| of the last residual                       */
    int iters;        /* residual evaluations performed                     */
    int converged;    /* 1 if max_r <= tol                                   */
    double seconds;   /* wall time of the solve                             */
    int switched_at;  /* MIXED: iteration of the BF16 -> BF16X6 switch, or -1 */
    int polished_at;  /* MIXED: iteration of the switch to defect correction, or -1 */
} dcsd_result;

/* dcsd_init -- create a context (Section II inputs of the method).
 *   out    : receives the context (NULL on error).
 *   d      : sizes.
 *   eps    : [n] orbital energies (informational; denominators are taken
 *            from the Fock diagonals).  May be NULL.
 *   fock_a, fock_b : [n][n] row-major Fock matrices of alpha and beta spin
 *            w.r.t. Phi_A (frozen-core contributions included).
 *   B      : [naux][n][n] DF factors, symmetric in the last two indices.
 *   mem_kind : whether eps/fock/B are host or device pointers; the library
 *            copies them.
 *   stream : cudaStream_t every call of this context enqueues on (NULL =
 *            legacy default stream).
 * Allocates the device memory of the FP64 residual and energy (device
 * pointers).  Everything else a call may need -- the tensor-core operand
 * buffers and FP32 accumulator of the BF16* precisions, the DIIS history
 * of dcsd_solve, the defect vector of the MIXED solve, the staging buffers
 * of host-memory (mem_kind HOST) calls -- is allocated by dcsd_reserve
 * ahead of time, or else by the first call that needs it (grow-only, kept
 * until dcsd_destroy).  dcsd_vjp and dcsd_lambda allocate their recorded
 * intermediates for the duration of the call.
 * Errors: INVALID_ARG (sizes < bounds, NULL pointers), OOM, CUDA, NO_DEVICE. */
dcsd_status dcsd_init(dcsd_ctx** out, const dcsd_dims* d, const double* eps,
                      const double* fock_a, const double* fock_b,
                      const double* B, int mem_kind, void* stream);

/* dcsd_reserve -- allocate now every device buffer that later calls of
 * this context would otherwise allocate on first use: dcsd_residual and
 * dcsd_energy at `precision` (DCSD_PREC_MIXED: the BF16 and BF16X6
 * residuals and the defect vector of the MIXED solve), dcsd_solve with up
 * to diis_n DIIS vectors (0: the two vectors of a Jacobi-only solve), and,
 * if host_staging is 1, the device staging of mem_kind HOST calls.  After
 * it, those calls allocate nothing (so that no allocation happens in the
 * middle of a solve, and memory use is known up front); device memory is
 * not released before dcsd_destroy.  The tensor-core buffers are sized by
 * running one CCSD residual at zero amplitudes in each of those precisions
 * (their sizes depend only on the dimensions); the context's amplitude
 * buffers are overwritten.  Synchronises the context stream.  Not part of
 * the paper's method: memory management of this library.
 * Errors: INVALID_ARG (bad precision, diis_n outside 0..16, host_staging
 * not 0/1), OOM, CUDA, TIMEOUT. */
dcsd_status dcsd_reserve(dcsd_ctx* ctx, int precision, int diis_n, int host_staging);

/* dcsd_residual -- one evaluation of the 2D residual (Eqs. 3-4).
 *   R = R^X(T) + M W with R^X the CCSD (method 0) or DCSD (method 1)
 *   single-reference residual; W = <B|H_N exp(T_A)|A>, which is R^X at the
 *   A->B double plus the products of the two internal singles with their
 *   R^X elements (zero in the CAS case); that element of R2ab is returned
 *   as zero.  dEA receives Delta E_A (Eq. 2).
 *   Fixed-reference methods (2..5): R = R^X(T) with the A->B amplitude at
 *   its fixed value and no M W terms; W receives R^X at the fixed
 *   excitation (not an equation of the method), whose R2ab element is
 *   returned as zero; dEA receives the FR energy.
 *   T* inputs and R* outputs use the layouts above; mem_kind says whether
 *   they are host (copied in and out inside the call, which then
 *   synchronises the stream) or device pointers (asynchronous on the
 *   context stream; W and dEA are still host doubles and the call
 *   synchronises before returning them).  Outputs may not alias inputs.
 *   precision: DCSD_PREC_FP64, _BF16, _BF16X3 or _BF16X6.
 * Errors: INVALID_ARG, CUDA, NUMERIC (NaN/Inf in R). */
dcsd_status dcsd_residual(dcsd_ctx* ctx, int ref, int method, int precision,
                          int mem_kind,
                          const double* T1a, const double* T1b,
                          const double* T2aa, const double* T2bb,
                          const double* T2ab,
                          double* R1a, double* R1b, double* R2aa,
                          double* R2bb, double* R2ab,
                          double* W, double* dEA);

/* dcsd_energy -- Delta E_A (Eq. 2) and W for the amplitudes T (same layout
 * and mem_kind rules as dcsd_residual; FP64).  W needs the doubles residual
 * element of the A->B excitation, so this runs one FP64 residual. */
dcsd_status dcsd_energy(dcsd_ctx* ctx, int ref, int method, int mem_kind,
                        const double* T1a, const double* T1b,
                        const double* T2aa, const double* T2bb,
                        const double* T2ab, double* dEA, double* W);

/* dcsd_solve -- converge the 2D amplitude equations on the GPU (Jacobi
 * steps with Fock-diagonal denominators + Pulay DIIS, all FP64 vector
 * algebra on the device).  T* are in/out (initial guess if
 * opts->use_guess, converged amplitudes on return), mem_kind as above.
 * Every iteration is one residual evaluation followed by one update; the
 * loop stops before the update once max|R| <= tol.  Returns NOT_CONVERGED
 * if maxiter is reached (T then holds the amplitudes after the last update,
 * *res the figures of the last residual). */
dcsd_status dcsd_solve(dcsd_ctx* ctx, const dcsd_solve_opts* opts, int mem_kind,
                       double* T1a, double* T1b, double* T2aa, double* T2bb,
                       double* T2ab, dcsd_result* res);

/* dcsd_heff -- the 2x2 effective Hamiltonian of the two references (Eq. 2
 * and the text after Eq. 4): H = [[dEA, W], [W, dEA]] (row-major H[4]),
 * its eigenvalues in ascending order evals[2], and *singlet_index, the
 * position of the singlet dEA + W in evals.  Pure host arithmetic. */
dcsd_status dcsd_heff(double dEA, double W, double* H, double* evals,
                      int* singlet_index);

/* dcsd_destroy -- free the context and all its device memory (NULL ok). */
dcsd_status dcsd_destroy(dcsd_ctx* ctx);

/* dcsd_last_error -- human-readable message of the last failed call of
 * ctx (or of the last failed dcsd_init when ctx is NULL). */
const char* dcsd_last_error(const dcsd_ctx* ctx);

/* dcsd_kernel_launches -- number of kernels this context has launched since
 * creation (diagnostics / benchmark accounting). */
long long dcsd_kernel_launches(const dcsd_ctx* ctx);

/* Kernel classes reported by dcsd_profile. */
typedef enum {
    DCSD_PROF_LADDER = 0,   /* tcgen05 GEMMs of the particle-particle ladder    */
    DCSD_PROF_TC_OTHER = 1, /* other tcgen05 GEMMs (ring, DF builds, ...)       */
    DCSD_PROF_PACK = 2,     /* BF16 operand packing                             */
    DCSD_PROF_FP64 = 3,     /* FP64 CUDA-core contractions                      */
    DCSD_PROF_NCLASS = 8
} dcsd_prof_class;

/* dcsd_profile -- device-time accounting of the context's kernels, measured
 * with CUDA events recorded on the context stream around every launch of
 * the classes above while enabled.
 *   enable : 1 start/continue recording, 0 stop.
 *   reset  : 1 clears the accumulated figures before (re)enabling.
 *   ms, launches : if non-NULL, arrays of DCSD_PROF_NCLASS receiving the
 *            summed device milliseconds and launch counts per class since
 *            the last reset (the call synchronises the stream to read them).
 * Errors: INVALID_ARG (NULL ctx), CUDA. */
dcsd_status dcsd_profile(dcsd_ctx* ctx, int enable, int reset, double* ms,
                         long long* launches);

/* dcsd_vjp -- vector-Jacobian product of the residual (reverse mode).
 * For the residual R(T) of dcsd_residual (same ref, method, precision) with outputs
 * (R1a, R1b, R2aa, R2bb, R2ab, dE_A, W), returns for given cotangents
 * (R_bar, dEA_bar, W_bar) the gradients of
 *     <R_bar, R(T)> + dEA_bar * dE_A(T) + W_bar * W(T)
 * with respect to the stored amplitude arrays (every element, as stored;
 * T2aa and T2bb are read as full arrays), the DF factors B and the two Fock
 * matrices of dcsd_init (2D methods 0 and 1 only).  The paper has no counterpart; this is the
 * derivative of the Section II residual used for the Lambda equations and
 * the response density of dcsd_lambda.
 *   T1a .. T2ab       : amplitudes, layout of this header.
 *   R1a_bar .. R2ab_bar : residual cotangents, same layouts; all five NULL
 *                       means zero.
 *   dEA_bar, W_bar    : cotangents of dE_A and W.
 *   T1a_bar .. T2ab_bar : out, gradients, same layouts.
 *   B_bar             : out or NULL, [naux][n][n] (both triangles: the
 *                       gradient with respect to the array as stored).
 *   fock_a_bar, fock_b_bar : out or NULL, [n][n].
 * precision: DCSD_PREC_FP64 (CUDA cores) or a tensor-core precision, in
 * which the forward and the adjoint contractions run on the tensor cores
 * with that operand split (the adjoint of a BF16X6 residual is accurate to
 * its FP32-class accuracy).
 * Pointers are host or device memory according to mem_kind.  The call runs
 * the residual once while recording its operations and then their
 * adjoints; the integrals of the particle-particle ladder and of its T1
 * correction are rebuilt in the reverse sweep, not stored.  Other intermediates are kept in device memory
 * for the duration of the call (about 25 doubly-sized amplitude arrays).
 * Errors: INVALID_ARG, OOM, CUDA. */
dcsd_status dcsd_vjp(dcsd_ctx* ctx, int ref, int method, int precision, int mem_kind,
                     const double* T1a, const double* T1b, const double* T2aa,
                     const double* T2bb, const double* T2ab,
                     const double* R1a_bar, const double* R1b_bar, const double* R2aa_bar,
                     const double* R2bb_bar, const double* R2ab_bar,
                     double dEA_bar, double W_bar,
                     double* T1a_bar, double* T1b_bar, double* T2aa_bar,
                     double* T2bb_bar, double* T2ab_bar,
                     double* B_bar, double* fock_a_bar, double* fock_b_bar);

/* dcsd_lambda -- Lambda equations and response density of one state.
 * With E = dE_A + state * W (state +1: the singlet of dcsd_heff's phase
 * convention, -1: the triplet) and the Lagrangian
 *     L(T, Lambda) = E(T) + sum_q Lambda_q R_q(T)
 * over the residual elements of dcsd_residual, solves dL/dT = 0 for Lambda
 * at converged amplitudes T (Jacobi steps with the amplitude denominators
 * and DIIS; each iteration is one reverse sweep of the recorded FP64
 * residual, see dcsd_vjp), and returns the response density
 *     gamma^sigma_pq = dL/df^sigma_pq
 * (the gradient with respect to the Fock matrices of dcsd_init as stored;
 * contract its symmetric part with symmetric perturbations).  By
 * stationarity, dE/df along any perturbation of f equals <gamma, df> once
 * T and Lambda are converged.  The paper has no counterpart; this is the
 * first-order property machinery of the Section II energies.
 *   o          : method (0 or 1), ref, maxiter, diis_n, tol (on max |dL/dT| over the
 *                independent amplitudes), use_guess (Lambda in L* is the
 *                guess); precision must be DCSD_PREC_FP64.
 *   T1a..T2ab  : converged amplitudes (dcsd_solve), layout of this header.
 *   L1a..L2ab  : in/out Lambda, same layouts; same-spin doubles
 *                antisymmetric, the A->B double element 0.
 *   rdm_a, rdm_b : out or NULL, [n][n].
 *   res        : dEA, W, E_S, E_T at T, iters, converged, max_r = final
 *                max |dL/dT|, seconds.
 * Pointers are host or device memory according to mem_kind.
 * Errors: INVALID_ARG, OOM, CUDA, NUMERIC, NOT_CONVERGED (outputs hold the
 * last iterate). */
dcsd_status dcsd_lambda(dcsd_ctx* ctx, const dcsd_solve_opts* o, int state, int mem_kind,
                        const double* T1a, const double* T1b, const double* T2aa,
                        const double* T2bb, const double* T2ab,
                        double* L1a, double* L1b, double* L2aa, double* L2bb, double* L2ab,
                        double* rdm_a, double* rdm_b, dcsd_result* res);

/* dcsd_selftest_conversions -- checks, on the current device, the FP64 <->
 * FP32 conversions that the tensor-core precision modes perform on the
 * integer units (IEEE 754 binary64/binary32, round to nearest even) against
 * the hardware conversions: every binary32 value to binary64, and 2^28
 * binary64 patterns covering every exponent with exact ties, near-ties and
 * random fractions to binary32.  NaN results compare equal to any NaN.  Not
 * part of the paper's method: a check of this library's arithmetic.
 *   stream     : cudaStream_t the kernels run on (synchronised before return).
 *   mismatches : host pointer receiving the number of differing results.
 * Errors: INVALID_ARG (NULL mismatches), NO_DEVICE, OOM, CUDA. */
dcsd_status dcsd_selftest_conversions(void* stream, long long* mismatches);

/* dcsd_coupling_host -- the two-determinant coupling coefficients
 * c_q = <Phi_q| exp(T_other) |Phi_other> of the M.W terms (Section II,
 * Eqs. 3-4: c_ia and c_ijab, with T_other the amplitudes of this frame with
 * alpha and beta exchanged), evaluated on the host from the same term
 * tables that the device kernels use (derived by excitation algebra on
 * occupation strings).  A diagnostic of the table derivation: it needs no
 * context and no GPU.
 *   ref        : 0 (Phi_A) or 1 (Phi_B), the frame of the amplitudes and q.
 *   n_c, n_v   : core orbitals and external virtuals (1..64 external, at
 *                most 64 core).
 *   T1a .. T2ab: host arrays, amplitude layout of this header.
 *   c1a .. c2ab: host arrays (same layouts) receiving c_q.  Same-spin
 *                elements with i == j or a == b and the A->B element are 0.
 * Errors: INVALID_ARG (bad ref or sizes, NULL pointer, or a table the
 * derivation rejects). */
dcsd_status dcsd_coupling_host(int ref, int n_c, int n_v, const double* T1a, const double* T1b,
                               const double* T2aa, const double* T2bb, const double* T2ab, double* c1a,
                               double* c1b, double* c2aa, double* c2bb, double* c2ab);

/* dcsd_einsum_host -- C = beta * C + alpha * einsum(spec)(A, B) on the host,
 * executed from the batched-GEMM plan (batch, row, column and contracted
 * modes, with adjacent modes merged) that the device contractions of this
 * library use for the same spec and views.  A diagnostic of the planner: it
 * needs no context and no GPU.
 *   spec               : "ab,bc->ac" form, one letter per mode; a letter in
 *                        A and B but not C is summed; in all three, batched.
 *   A, B, C            : host arrays (FP64); C is read only if beta != 0.
 *   rank_x, size_x, stride_x : view of each operand, strides in elements.
 * Errors: INVALID_ARG (NULL pointer, rank above 8, a spec the planner
 * rejects: rank or size mismatch, repeated letter in one operand, a letter
 * summed in one operand only, more than 4 unmergeable modes of one kind). */
dcsd_status dcsd_einsum_host(const char* spec, double alpha, const double* A, int rank_a,
                             const long* size_a, const long* stride_a, const double* B, int rank_b,
                             const long* size_b, const long* stride_b, double beta, double* C, int rank_c,
                             const long* size_c, const long* stride_c);

/* dcsd_energy_noalloc -- Delta E_A, the value dcsd_energy returns as dEA,
 * for callers that cannot allocate device memory: code that is
 * capturing a CUDA graph, that hands all device memory to its own pool
 * allocator, or that must keep a fixed footprint.  The paper has no
 * counterpart; this is a service of the library.
 *   n_c, n_v, naux, ref : as for dcsd_init / dcsd_residual.
 *   fock_a, fock_b, B   : device pointers, layouts of dcsd_init.
 *   T1a .. T2ab         : device pointers, amplitude layout of this header.
 *   dEA                 : device pointer receiving one double.
 *   stream              : cudaStream_t the two kernels are enqueued on; the
 *                         call does not synchronise it.
 * Allocates nothing: its only working memory is a fixed device array that
 * is part of the library (8192 doubles, one partial sum per spin block and
 * occupied pair), so n_c + 1 must not exceed 52 (else INVALID_ARG).  The
 * array is shared by all calls and keeps the last call's contents: calls
 * that overlap on the GPU race and must be serialised by the caller.  The
 * first call on a device looks up the array's device address (no
 * allocation); make that first call before any stream capture begins.
 * Errors: INVALID_ARG (NULL pointer, sizes beyond the limit), NO_DEVICE,
 * CUDA (launch failure). */
dcsd_status dcsd_energy_noalloc(int n_c, int n_v, int naux, int ref,
                                const double* fock_a, const double* fock_b,
                                const double* B, const double* T1a,
                                const double* T1b, const double* T2aa,
                                const double* T2bb, const double* T2ab,
                                double* dEA, void* stream);

/* ---------------------------------------------------------------------------
 * FCIDUMP input.  The paper's calculations read their integrals from
 * FCIDUMP files written after the ROHF or 2D-SCF step (Section III,
 * computational details).  Format: the namelist header &FCI NORB, NELEC,
 * MS2, ORBSYM, ISYM &END, then lines "value i j k l" (1-based): (ij|kl)
 * (chemists' notation, one of the eight equivalent permutations), h_ij
 * (k = l = 0), orbital energies (j = k = l = 0, ignored) and the core
 * energy (all zero).  Spin-restricted orbitals only (IUHF files are
 * refused).  The host code keeps the four-index integrals as a dense array,
 * so NORB is limited to 160.  The open-shell determinant Phi_A doubly
 * occupies the first (NELEC - 2) / 2 orbitals and singly occupies the next
 * two, t (alpha) and u (beta); MS2 must be 0.
 * ------------------------------------------------------------------------- */
typedef struct {
    int norb, nelec, ms2;     /* from the header                                 */
    int n_frozen;             /* frozen core orbitals folded into h              */
    int n_c, n_v, naux;       /* dimensions of the context (naux = Cholesky rank) */
    double e_core;            /* core energy incl. the frozen-core contribution  */
    double e_ref;             /* <Phi_A|H|Phi_A>, total reference energy         */
    double chol_max_error;    /* bound on |(pq|rs) - sum_L B_pq^L B_rs^L|        */
} dcsd_fcidump_info;

/* dcsd_fcidump_header -- NORB, NELEC and MS2 of an FCIDUMP file (host).
 * Errors: INVALID_ARG (NULL pointer, unreadable file, no &FCI header, NORB
 * outside 1..160, IUHF file); dcsd_fcidump_error() has the message. */
dcsd_status dcsd_fcidump_header(const char* path, int* norb, int* nelec, int* ms2);

/* dcsd_fcidump_read -- the integrals of an FCIDUMP file (host):
 *   h     : out, [norb][norb] one-electron integrals, symmetric;
 *   eri   : out, [norb]^4 two-electron integrals (pq|rs) with all eight
 *           permutations of every listed element filled; absent ones 0;
 *   ecore : out, the core energy.
 * norb must equal the header's NORB.  Errors: INVALID_ARG (as above, a
 * malformed line, an index outside 0..NORB). */
dcsd_status dcsd_fcidump_read(const char* path, int norb, double* h, double* eri, double* ecore);

/* dcsd_cholesky_host -- pivoted Cholesky factorisation of the integral
 * matrix V[(pq),(rs)] = (pq|rs) (Beebe and Linderberg, 1977; host): factors
 * B[L][p][q], L < *rank, with |(pq|rs) - sum_L B^L_pq B^L_rs| <= tol for
 * every element.  The paper uses full four-index integrals; this exact
 * factorisation lets them enter the engine in the factorised form its
 * kernels use in place of density fitting.
 *   n        : orbitals (<= 160); eri : [n]^4 (pq|rs), symmetric as above.
 *   tol      : threshold on the remaining diagonal, > 0 (e.g. 1e-12).
 *   max_rank : capacity of B in factors (n (n + 1) / 2 always suffices).
 *   B        : out, [max_rank][n][n].  rank : out.  max_diag_left : out or
 *              NULL, the largest remaining diagonal element (the error bound).
 * Errors: INVALID_ARG. */
dcsd_status dcsd_cholesky_host(int n, const double* eri, double tol, int max_rank, double* B, int* rank,
                               double* max_diag_left);

/* dcsd_fcidump_prepare -- everything dcsd_init needs from an FCIDUMP file
 * (host): frozen-core folding of the first n_frozen orbitals into h and the
 * core energy, the Fock matrices of Phi_A over the correlated orbitals,
 * f^s_pq = h'_pq + sum_{k in Phi_A} [(pq|kk) - delta(s_k, s) (pk|kq)], the
 * Cholesky factors of the correlated integrals (threshold chol_tol) and the
 * reference energy.  Call first with NULL arrays to learn the sizes in
 * *info (n = n_c + 2 + n_v, naux), then with fock_a, fock_b [n][n] and B
 * [naux][n][n].  Errors: INVALID_ARG (file errors as above, MS2 != 0, odd
 * NELEC, n_frozen outside 0..(NELEC-2)/2, no virtual orbital). */
dcsd_status dcsd_fcidump_prepare(const char* path, int n_frozen, double chol_tol, dcsd_fcidump_info* info,
                                 double* fock_a, double* fock_b, double* B);

/* dcsd_init_fcidump -- dcsd_fcidump_prepare followed by dcsd_init (host
 * inputs) on `stream`.  stored_ladder 1 also keeps the four-index (ac|bd)
 * of the virtual orbitals (t, u and the external ones) on the device, and
 * the FP64 residual then takes its particle-particle ladder from them
 * instead of from the factors (a check of the factorised ladder; the
 * tensor-core precisions and the reverse mode always use the factors).
 * info : out or NULL.  Errors: those of both calls; OOM for the stored
 * integrals. */
dcsd_status dcsd_init_fcidump(dcsd_ctx** out, const char* path, int n_frozen, double chol_tol, int stored_ladder,
                              void* stream, dcsd_fcidump_info* info);

/* dcsd_fcidump_error -- message of the last failed FCIDUMP call (host,
 * process-wide). */
const char* dcsd_fcidump_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DCSD_H */
