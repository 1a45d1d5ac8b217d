/*
 * fmmcph -- fast multipole Coulomb solver for lambda-dynamics constant pH,
 * B300 (sm_103a) native.  C ABI.
 *
 * What one evaluation computes (arXiv 2410.01626):
 *   Sites k = 0..K-1 each carry a titration coordinate lambda_k.  Atom i of
 *   site s(i) carries the charge
 *       q_i = qA_i + lambda_{s(i)} (qB_i - qA_i)
 *   (Sec. 2.1, Eq. 1: the Hamiltonian is interpolated linearly between the
 *   forms A and B, and the forms differ only in their charges; atoms outside
 *   every site have s(i) = -1 and q_i = qA_i).  The Coulomb solver of
 *   Sec. 2.6 (a fast multipole method) then returns
 *       E             = 1/2 k_e sum_i q_i phi_i
 *       F_i           = -dE/dx_i = -k_e q_i grad phi_i
 *       dV/dlambda_k  = dE/dlambda_k = k_e sum_{i: s(i)=k} (qB_i - qA_i) phi_i
 *   with phi_i = sum_{j != i} q_j / |x_i - x_j| in an open cube, or the
 *   tinfoil Ewald potential (uniform neutralising background) in a periodic
 *   cube.  dV/dlambda_k is the force on the lambda particle that drives the
 *   titration (Sec. 2.1, F_lambda = -dH/dlambda).
 *   The user-facing knobs are the multipole order p and the tree depth
 *   (Sec. 2.9, minimal mdp figure: p = 8, depth 2 for an 8 nm box).
 *
 * Units: x in nm, q in e, k_e defaults to 138.935458 kJ mol^-1 nm e^-2, so E
 * and dV/dlambda are in kJ/mol and F in kJ mol^-1 nm^-1.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers unless the name ends in _host.
 *     They are owned by the caller; the library never frees them.
 *   - Calls are asynchronous on the CUDA stream passed as `stream` (a
 *     cudaStream_t; NULL = the legacy default stream).  A handle must not be
 *     used from two host threads at once.
 *   - Argument errors are detected on the host, synchronously, and returned
 *     as a status code; nothing is launched in that case.  Conditions only
 *     the device can see (an atom outside an open box, a site index >= K)
 *     set bits in a device status word, read with fmm_status_word().
 *     The library never traps the GPU.
 */
#ifndef FMMCPH_H
#define FMMCPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = 1,     /* invalid argument (null pointer, size, range)       */
    FMM_ERR_DOMAIN = 2,  /* device status: an atom outside an open box         */
    FMM_ERR_CUDA = 3,    /* a CUDA runtime call failed                          */
    FMM_ERR_OOM = 4,     /* device allocation failed                            */
    FMM_ERR_TIMEOUT = 5, /* a bounded device wait gave up                       */
    FMM_ERR_STATE = 6    /* call order violated (e.g. eval before charges)      */
} fmm_status;

/* device status word bits (fmm_status_word) */
#define FMM_DEV_DOMAIN 1   /* atom outside [origin, origin + edge] of an open box */
#define FMM_DEV_SITE 2     /* site index >= K (atom treated as not in a site)    */
#define FMM_DEV_TIMEOUT 4  /* bounded wait expired                               */
#define FMM_DEV_BOUNDS 8   /* an index check failed (bounds-checked build only)   */

/* fmm_build_flags bits */
#define FMM_BUILD_BOUNDS_CHECK 1 /* built with -DFMM_BOUNDS_CHECK (libfmmcph_checked.so) */

typedef enum {
    FMM_FP32 = 0,        /* every stage in FP32 on CUDA cores (root/lattice FP64) */
    FMM_MIXED_TF32 = 1,  /* M2L on tcgen05 tensor cores in TF32, FP32 accumulate  */
    FMM_MIXED_3XTF32 = 2, /* M2L as three TF32 products (split operands)          */
    FMM_MIXED_3XBF16 = 3, /* M2L as three BF16 products hi*hi + hi*lo + lo*hi of
                             split operands (about 16 significant bits, twice the
                             tensor rate of TF32), FP32 accumulate                  */
    FMM_MIXED_FP16 = 4    /* M2L in FP16 on the tensor cores, FP32 accumulate: the
                             input coefficients of degrees 0..3 as three products of
                             split hi/lo operands (about 22 bits), all higher degrees
                             as one product (11 bits) -- the far field's monopole and
                             dipole parts keep full accuracy at about 0.4 of the
                             3xBF16 tensor work                                      */
} fmm_precision;

typedef struct {
    double origin[3]; /* lower corner, nm          */
    double edge;      /* cube edge length L, nm > 0 */
} fmm_box;

/* How the energy depends on lambda within a site (Sec. 2.1, Eq. 1).
 * CHARGE: the charges are interpolated, q_i = qA_i + lambda (qB_i - qA_i),
 *   and E is the Coulomb energy of q(lambda).
 * HAMILTONIAN: the Hamiltonian is interpolated; pairs in different sites (and
 *   all pairs with other atoms) are the same as above, pairs i, j within one
 *   site k differ by lambda_k (1 - lambda_k) dq_i dq_j psi(r_ij), where psi is
 *   the pair potential of the box (1/r open; the periodic pair potential with
 *   its self-image term for i = j).  E is then linear in every lambda_k, and
 *   F and dV/dlambda include the correction.  phi (fmm_eval) stays the
 *   potential of q(lambda). */
typedef enum { FMM_INTERP_CHARGE = 0, FMM_INTERP_HAMILTONIAN = 1 } fmm_interpolation;

typedef struct {
    int precision;      /* fmm_precision                           */
    double coulomb_k;   /* k_e; <= 0 selects 138.935458             */
    int interpolation;  /* fmm_interpolation                       */
    /* Kernel tiles (results are the same for every choice; the autotuner picks them by timing).
     * m2l_tile_rows: rows of the tensor-core M2L's per-CTA tile (the MMA's N): 128, 160, 192,
     *   224 or 256; 0 selects 192.
     * p2p_leaves_per_block: target leaves (one warp each) per near-field block: 1, 2 or 4; 0
     *   selects 1.
     * Other values return FMM_ERR_ARG. */
    int m2l_tile_rows;
    int p2p_leaves_per_block;
    int reserved[5];    /* must be zero                             */
} fmm_options;

typedef struct fmm_handle fmm_handle;

/* Create a solver for one cubic box.
 *   periodic: 0 = open boundary, 1 = periodic (tinfoil, neutralising background)
 *   p:        maximum expansion degree, 1 <= p <= FMM_MAX_P
 *   depth:    octree depth, 8^depth leaves; 0 <= depth <= 7
 *   opt:      may be NULL (FP32, default k_e)
 * The mixed precisions (tensor-core M2L) need p <= 10 and depth <= 5; other
 * combinations return FMM_ERR_ARG rather than fall back to another precision
 * (FMM_FP32 takes every p and depth).
 * Builds the translation operators on the host in FP64 (the periodic lattice
 * operator by projecting the Ewald remainder onto solid harmonics) and
 * uploads them.  Synchronous.  Returns FMM_ERR_ARG, FMM_ERR_OOM or
 * FMM_ERR_CUDA on failure, with *out set to NULL. */
#define FMM_MAX_P 14
fmm_status fmm_create(const fmm_box* box, int periodic, int p, int depth, const fmm_options* opt,
                      fmm_handle** out);

/* Set the atoms' charge forms and the site map, and lambda.
 *   qA, qB:  [n_atoms] float, charges of forms A and B (e)
 *   site:    [n_atoms] int32, site index in [0, n_sites) or -1
 *   lambda:  [n_sites] float (may be NULL when n_sites == 0)
 * The arrays are copied (stream-ordered), so the caller may reuse them after
 * the copy has executed.  Grows the handle's device buffers when n_atoms
 * exceeds the previous capacity (synchronous allocation).  n_atoms >= 0,
 * n_sites >= 0.  Site indices >= n_sites set FMM_DEV_SITE on the next eval. */
fmm_status fmm_set_charges(fmm_handle* h, int n_atoms, int n_sites, const float* qA,
                           const float* qB, const int32_t* site, const float* lambda,
                           void* stream);

/* Sites with two lambda coordinates over four charge forms (Sec. 2.1, Eq. 2:
 * protonation lambda_p and tautomer lambda_t):
 *   q_i = (1 - lp)[(1 - lt) qA_i + lt qB_i] + lp[(1 - lt) qC_i + lt qD_i]
 * for atoms of a site; other atoms keep qA_i.  A site without tautomers has
 * qB = qA and qD = qC (its lt derivative is then 0).
 *   qA .. qD: [n_atoms] float (device), the four forms
 *   site:     [n_atoms] int32, site index in [0, n_sites) or -1
 *   lambda:   [2 n_sites] float (device): lp_0, lt_0, lp_1, lt_1, ...
 * Otherwise as fmm_set_charges.  Until the next fmm_set_charges, every
 * lambda and dV/dlambda array of this handle (fmm_set_lambda,
 * fmm_bind_lambda, fmm_eval, fmm_eval_host, fmm_adjoint4, fmm_lambda_step)
 * has 2 n_sites entries in this order; with Hamiltonian interpolation the
 * intra-site correction uses the covariance of the forms' charges. */
fmm_status fmm_set_charges4(fmm_handle* h, int n_atoms, int n_sites, const float* qA,
                            const float* qB, const float* qC, const float* qD,
                            const int32_t* site, const float* lambda, void* stream);

/* Replace lambda ([n_sites] float, device), stream-ordered copy. */
fmm_status fmm_set_lambda(fmm_handle* h, const float* lambda, void* stream);

/* Use the caller's device buffer for lambda from now on (no copy): each
 * fmm_eval reads lambda at launch time from `lambda` ([n_sites] float).
 * Lets a device-side lambda integrator feed the solver with no host call
 * between steps.  Pass NULL to go back to the handle's own copy. */
fmm_status fmm_bind_lambda(fmm_handle* h, const float* lambda);

/* One evaluation.
 *   x:          [n_atoms][3] float positions (nm), input order
 *   E:          [1] double, energy (kJ/mol)
 *   F:          [n_atoms][3] float forces, input order (may be NULL)
 *   dVdlambda:  [n_sites] float (may be NULL)
 *   phi:        [n_atoms] float, k_e * potential at each atom (kJ/mol/e),
 *               input order (may be NULL)
 * Stream-ordered; all outputs are complete when the stream reaches the end
 * of the call.  Returns FMM_ERR_STATE before fmm_set_charges.
 * Evaluations of one handle on different streams are ordered by the handle:
 * an evaluation on a stream other than the previous evaluation's waits for
 * the end of that evaluation's kernels (not for later work on its stream),
 * except inside a capture by the caller.
 * When the same five pointers come again within the handle's last two eager
 * evaluations, the evaluation is captured into a CUDA graph owned by the
 * handle (on a private stream), and later calls with those pointers replay
 * it on `stream`; the handle keeps the graphs of the two most recent pointer
 * sets (so two sets used in turn both replay).  The kernels and the results
 * are those of launching them one by one.  A graph reads the buffers at
 * replay, so positions and lambda written in place (or with fmm_set_lambda)
 * are seen; fmm_set_charges*, fmm_bind_lambda, fmm_set_profiling and
 * fmm_set_wait_limit discard the graphs.  While profiling, or when `stream`
 * is being captured by the caller, the kernels are launched one by one (and
 * so join the caller's capture). */
fmm_status fmm_eval(fmm_handle* h, const float* x, double* E, float* F, float* dVdlambda,
                    float* phi, void* stream);

/* Makes `stream` wait for the end of the kernels of the handle's last
 * evaluation (fmm_eval, fmm_eval_host, fmm_eval_host_async), not for the
 * result copies that fmm_eval_host(_async) enqueues after them: work the
 * caller enqueues on `stream` afterwards runs after that evaluation, beside
 * its copies.  Nothing to do when no evaluation has been enqueued, or the
 * last one was on `stream` or inside a capture.  FMM_ERR_ARG for a null
 * handle. */
fmm_status fmm_stream_wait_eval(fmm_handle* h, void* stream);

/* The same evaluation with HOST buffers: copies x_host to the device, runs
 * fmm_eval (on the handle's own device staging buffers, so from the second
 * call on as a graph replay) and copies E, F and dV/dlambda back, then
 * synchronises `stream`.
 * For page-locked host buffers the copies are asynchronous DMA.  Any output
 * pointer may be NULL. */
fmm_status fmm_eval_host(fmm_handle* h, const float* x_host, double* E_host, float* F_host,
                         float* dVdlambda_host, void* stream);

/* fmm_eval_host without the final synchronisation, for callers that keep several
 * evaluations in flight: enqueues the copy of x_host to the device, the evaluation and the
 * copies of E, F and dV/dlambda back, and returns.  The results are in the host buffers once
 * `stream` has reached the end of the call (cudaStreamSynchronize, or an event recorded
 * after it); until then the caller must keep the buffers and leave x_host unchanged.
 * Consecutive calls use two device staging sets in turn: a call's position copy runs on the
 * handle's own copy stream as soon as its set's previous use has finished, so with
 * page-locked buffers it overlaps the previous call's evaluation.  Calls that alternate two
 * streams also overlap a call's result copies with the next call's evaluation (the handle
 * orders the evaluations, see fmm_eval); give each call in flight its own output buffers.
 * When `stream` is being captured the copy runs on `stream` itself. */
fmm_status fmm_eval_host_async(fmm_handle* h, const float* x_host, double* E_host, float* F_host,
                               float* dVdlambda_host, void* stream);

/* Page-locked host memory for the buffers of fmm_eval_host (not part of the
 * method; a convenience for callers).  Copies between this memory and the
 * device are asynchronous DMA.  They run at the PCIe rate (6 MB in 0.12 ms
 * each way on the B300 hosts measured here) while the CPU caches hold none of
 * the buffer's lines; a buffer the CPU has just written or read runs several
 * times slower on those hosts (a 6 MB host-to-device copy from a buffer
 * written by the CPU took 0.5-1.3 ms, and write-combined memory did no
 * better there).  fmm_host_alloc writes the
 * address to *out (NULL on failure) and returns FMM_ERR_ARG for bytes == 0 or
 * out == NULL, FMM_ERR_OOM when the allocation fails.  Free with
 * fmm_host_free (NULL is ignored). */
fmm_status fmm_host_alloc(size_t bytes, void** out);
void fmm_host_free(void* p);

/* Adjoint of E(x, qA, qB, lambda) for reverse-mode differentiation.
 *   gbar:       [1] double, dL/dE (device)
 *   F, phi:     outputs of the preceding fmm_eval (input order)
 *   grad_x:     [n_atoms][3] float, dL/dx = -F * gbar            (may be NULL)
 *   grad_qA:    [n_atoms] float, dL/dqA_i = phi_i (1 - lambda_s) * gbar
 *               (phi_i * gbar for atoms outside sites)           (may be NULL)
 *   grad_qB:    [n_atoms] float, dL/dqB_i = phi_i lambda_s * gbar (may be NULL)
 *   dVdlambda:  [n_sites] float from the same fmm_eval
 *   grad_lambda:[n_sites] float, dL/dlambda = dV/dlambda * gbar   (may be NULL)
 * E is quadratic in the charges, so dE/dq_i = k_e phi_i (the phi returned by
 * fmm_eval already includes k_e). */
fmm_status fmm_adjoint(fmm_handle* h, const double* gbar, const float* F, const float* phi,
                       const float* dVdlambda, float* grad_x, float* grad_qA, float* grad_qB,
                       float* grad_lambda, void* stream);

/* Adjoint for four-form sites (after fmm_set_charges4): dL/dq^X_i =
 * (phi_i + k_e g_X,i) w_X(lp, lt) * gbar for form X of a site atom (w_X its
 * bilinear weight; g_X,i the Hamiltonian-interpolation term, 0 otherwise),
 * dL/dqA_i = phi_i * gbar outside sites; grad_lambda and dVdlambda have
 * 2 n_sites entries.  Any output may be NULL.  FMM_ERR_STATE for two-form
 * sites (use fmm_adjoint), and fmm_adjoint returns FMM_ERR_STATE for
 * four-form sites. */
fmm_status fmm_adjoint4(fmm_handle* h, const double* gbar, const float* F, const float* phi,
                        const float* dVdlambda, float* grad_x, float* grad_qA, float* grad_qB,
                        float* grad_qC, float* grad_qD, float* grad_lambda, void* stream);

/* Copy the binning of the last fmm_eval into caller device buffers (any may
 * be NULL): key [n_atoms] uint32 Morton key of each atom's leaf (input
 * order), perm [n_atoms] uint32 (perm[s] = input index of the s-th atom in
 * leaf order; stable on (key, index)), start/count [8^depth] uint32. */
fmm_status fmm_get_binning(fmm_handle* h, uint32_t* key, uint32_t* perm, uint32_t* start,
                           uint32_t* count, void* stream);

/* Read and clear the device status word (FMM_DEV_* bits).  Synchronises
 * `stream` first.  In the bounds-checked build it also reads and clears the
 * library's index-check words: after a failed check it sets FMM_DEV_BOUNDS
 * and fmm_last_error names the source file and line of the first failure
 * (the words are per library, not per handle). */
fmm_status fmm_status_word(fmm_handle* h, int* device_status, void* stream);

/* How this library was built: FMM_BUILD_* bits.  The bounds-checked build
 * (-DFMM_BOUNDS_CHECK) checks the data-dependent indices of its kernels
 * (leaf keys, sorted slots, permutation entries, leaf ranges, site atoms,
 * staged-buffer offsets, packed-box and operator indices) against their
 * extents; a failed check skips the access it guards and is reported
 * through fmm_status_word.  No GPU needed. */
int fmm_build_flags(void);

/* Per-stage device times of the last fmm_eval when profiling is enabled
 * (CUDA events; profiling mode launches kernel by kernel).  ms[0..n):
 *   0 binning, 1 P2M, 2 M2M: consecutive, from the start of the evaluation;
 *   3 root: the periodic root multipole, lattice operator and Q/D/T sums (0
 *     in an open box);
 *   4 M2L: the M2L of the levels on the internal chain stream (pack + MMA
 *     kernel; with the side branch below, the MMA kernel of the two finest
 *     levels only, after their pack and the wait for the near field);
 *   5 L2L: the L2L into the levels after the M2L of ms[4] (with the side
 *     branch, the wait for it and the L2L into the two finest levels);
 *   6 outputs: the wait for the chain, then L2P, F, phi, energy partials;
 *   7 final: E and dV/dlambda;
 *   8 near field (P2P): from the end of binning, on the eval's stream,
 *     concurrently with P2M .. M2M;
 *   9, 10: with the tensor-core M2L and tree levels below the two finest,
 *     a side branch forked after the M2M runs the M2L of those coarse levels
 *     (ms[9]: the MMA kernel, after their pack and the wait for the near
 *     field), then the root (ms[3]) and the L2L into the coarse levels
 *     (ms[10]), concurrently with ms[4]; 0 without it.
 * The chain and the side branch run on internal streams of the handle,
 * forked from and joined back to the eval's stream, so graph capture of
 * fmm_eval works.  Synchronises.  Returns the number of stages written (at
 * most 11). */
int fmm_stage_times(fmm_handle* h, float* ms, int n);
/* enable: 0 off, 1 per-stage events (the stages overlap as in an ordinary evaluation), 2 the
 * same with every stage run on the eval's stream one after the other, so that each stage's
 * time is that of its kernels alone; FMM_ERR_ARG otherwise. */
fmm_status fmm_set_profiling(fmm_handle* h, int enable);

/* Bounded device waits.  The tensor-core M2L kernel runs as a pipeline of warps (bulk-copy
 * producer, MMA issuer, accumulator drains) that wait on one another through shared-memory
 * barriers; the tensor-core M2M and L2L wait for their operator copies and MMAs, and every
 * near-field warp for the copies of its staged atoms.  Each such wait gives up after a limit
 * of `cycles` GPU clock cycles (<= 0 selects the default, about 2 s).  A CTA (or near-field
 * warp) whose wait expires stops issuing work, waits (with the default limit) for the copies
 * and MMAs it already issued, frees its tensor memory and returns; the evaluation then sets
 * FMM_DEV_TIMEOUT in the status word (its results are not valid) and the handle stays usable.
 * A small limit is a test of that path; no evaluation should need more than the default.
 * Discards the handle's evaluation graph. */
fmm_status fmm_set_wait_limit(fmm_handle* h, long long cycles);

/* Test hook for the bounded waits of kernels whose waits do not otherwise run out: in the
 * kernels named by `mask` the bulk copies are announced on their barriers but never issued,
 * so their waits expire after the handle's wait limit (fmm_set_wait_limit; set a short one)
 * and the evaluation sets FMM_DEV_TIMEOUT.  FMM_LOSE_TRANSLATE: the operator copies of the
 * tensor-core M2M and L2L (the mixed-precision forms; FMM_FP32 translates on CUDA cores);
 * FMM_LOSE_NEAR: the near field's staging copies of leaves that fit
 * the staging buffer.  0 restores normal evaluation.  Discards the handle's evaluation graph.
 * FMM_ERR_ARG for a null handle or other bits. */
#define FMM_LOSE_TRANSLATE 1
#define FMM_LOSE_NEAR 2
fmm_status fmm_inject_copy_loss(fmm_handle* h, int mask);

/* Allocation-failure injection, for tests of the out-of-memory paths: with n >= 1 the n-th
 * device allocation the library makes from now on (in any handle or thread) fails as if the
 * device were out of memory, and the call that made it returns FMM_ERR_OOM after releasing
 * what it had allocated; n = 0 switches the injection off.  Returns FMM_ERR_ARG for n < 0. */
fmm_status fmm_inject_alloc_failure(int n);

/* Number of kernel launches one fmm_eval issues with the current settings. */
int fmm_launches_per_eval(const fmm_handle* h);

/* Host-side operator construction, exposed for CPU tests of the host logic
 * (no GPU needed).  Writes the FP64 real-form operator of the given kind in
 * the library's normalised coefficient basis, nc x nc row-major, nc =
 * (p+1)^2:
 *   kind 0: M2L for source offset (o[0], o[1], o[2]) boxes, |o|_inf in 2..3
 *   kind 1: M2M child octant o[0] (0..7) -> parent
 *   kind 2: L2L parent -> child octant o[0]
 *   kind 3: periodic lattice operator (root multipole -> root local)
 * Returns FMM_OK or FMM_ERR_ARG. */
fmm_status fmm_host_operator(int kind, int p, const int* o, double* out);

/* Evaluate the normalised regular solid harmonics at u (real form, length
 * (p+1)^2) on the host -- the basis P2M and L2P use.  Test helper. */
fmm_status fmm_host_regular(int p, const double* u, double* out);

/* One Langevin (BAOAB) step of the lambda particles on the device, driven by the force
 * -dV/dlambda of the preceding fmm_eval (Sec. 2.1, Eq. 1; lambda particle of mass m, Sec. 2.7).
 *   lambda, velocity: [n_sites] float, updated in place; dVdlambda: [n_sites] float
 *   dt (ps), mass (u), gamma (1/ps), kT (kJ/mol); reflecting walls at lo < hi
 *   seed, step: counter-based Philox4x32-10 stream (reproducible, resumable from a step)
 *   first: nonzero on the first step (half kick)
 * With fmm_bind_lambda(h, lambda) the next fmm_eval uses the new charges directly, so an
 * eval + step loop runs without host involvement and can be captured in a CUDA graph. */
fmm_status fmm_lambda_step(int n_sites, float* lambda, float* velocity, const float* dVdlambda, double dt,
                           double mass, double gamma, double kT, unsigned long long seed,
                           unsigned long long step, int first, double lo, double hi, void* stream);

/* The lambda-side bias potential (Sec. 2.2) on one lambda coordinate: a double well of
 * cubic Hermite pieces, wells at a0 < a1, the central barrier at b = (a0 + a1) / 2,
 *   V(a0) = 0, V(b) = barrier, V(a1) = delta, zero slope at a0, b and a1,
 * each piece V_a + (V_b - V_a)(3 s^2 - 2 s^3), and harmonic walls kwall (l - a)^2 / 2
 * outside [a0, a1].  The pH potential (Eq. 4) enters through delta:
 * fmm_lambda_pfc returns the delta (partition function correction, Sec. 2.3) for which
 * the partition functions Z_prot = int_lo^b exp(-V / kT) (protonated, lambda near 0) and
 * Z_deprot = int_b^hi exp(-V / kT) satisfy Z_deprot / Z_prot = 10^(pH - pKa_ref), the free
 * energy of deprotonation ln(10) kT (pKa_ref - pH) of Eq. 4.  Sec. 2.3 integrates over
 * [0, 0.5] and [0.5, 1]: pass lo = 0, hi = 1 (with a0 = 0, a1 = 1).  Passing the reflecting
 * walls of fmm_lambda_step instead (lo = -0.1, hi = 1.1) makes the condition hold for the
 * population the dynamics samples, which the paper's integrals leave out.  Host FP64
 * (Gauss-Legendre quadrature, bisection).  Returns FMM_ERR_ARG for kT <= 0, a0 >= a1,
 * lo >= b, hi <= b, kwall < 0 or delta == NULL. */
fmm_status fmm_lambda_pfc(double pH, double pKa_ref, double barrier, double kT, double a0, double a1,
                          double kwall, double lo, double hi, double* delta);

/* fmm_lambda_step with the bias potential: the force on coordinate k is
 * -dV/dlambda_k - dV_dw/dlambda(lambda_k; bias[5k .. 5k+4] = a0, a1, barrier, delta,
 * kwall), evaluated at the current lambda.  bias: [n][5] float (device); NULL is the
 * unbiased step. */
fmm_status fmm_lambda_step_bias(int n, float* lambda, float* velocity, const float* dVdlambda,
                                const float* bias, double dt, double mass, double gamma, double kT,
                                unsigned long long seed, unsigned long long step, int first, double lo,
                                double hi, void* stream);

/* Batches of independent replicas (different sizes, boxes, depths, precisions).
 * fmm_batch_create takes n existing handles (charges already set; the batch does not own
 * them).  fmm_batch_eval evaluates every replica; x, E, F, dVdlambda are HOST arrays of n
 * DEVICE pointers (F, dVdlambda and their entries may be NULL).  The replicas run as
 * parallel branches of one CUDA graph, captured on the first call and re-captured whenever
 * a pointer changes; later calls are one graph launch on `stream`.  Each replica's result is
 * bitwise identical to its own fmm_eval. */
typedef struct fmm_batch fmm_batch;
fmm_status fmm_batch_create(int n, fmm_handle* const* handles, fmm_batch** out);
fmm_status fmm_batch_eval(fmm_batch* b, const float* const* x, double* const* E, float* const* F,
                          float* const* dVdlambda, void* stream);
void fmm_batch_destroy(fmm_batch* b);

/* Binning with no device allocation.  Some callers cannot call cudaMalloc: a host program
 * (an MD engine, for instance) that owns all of the GPU's memory through its own pool or a
 * fixed budget, or a loop that must not stall, since cudaMalloc may synchronise the device.
 * For them this call runs the binning step of fmm_eval (Morton keys, stable sort, leaf
 * ranges) without allocating: its sort scratch is a static device array inside the library.
 * The paper has no counterpart.
 *   box, periodic, depth: as for fmm_create (0 <= depth <= 7)
 *   n_atoms:  0 <= n_atoms <= FMM_NOALLOC_MAX_ATOMS, else FMM_ERR_ARG (nothing launched)
 *   x:        [n_atoms][3] float positions (device)
 *   key, perm:[n_atoms] uint32 outputs, start, count: [8^depth] uint32 outputs (device) -- the
 *             values fmm_get_binning returns after fmm_eval on the same positions
 *   status:   one device int or NULL; when given, FMM_DEV_DOMAIN is OR-ed into it if an atom
 *             lies outside an open box (such atoms are clamped into the boundary leaves).  The
 *             call only sets bits: the caller clears the word.
 * The scratch holds FMM_NOALLOC_MAX_ATOMS atoms (about 6.5 MB on every GPU that loads the
 * library, kept until the process exits).  The first call on a device looks up the array's
 * device address (with that device current) and caches it; make that first call before any
 * stream capture.  Every call uses the same array, and the array keeps the last call's
 * contents (nothing in it needs to start at zero), so calls that overlap on the GPU -- on
 * streams with no ordering between them -- race; calls on one stream are ordered.  No
 * device memory is allocated or freed. */
#define FMM_NOALLOC_MAX_ATOMS 524288
fmm_status fmm_binning_noalloc(const fmm_box* box, int periodic, int depth, int n_atoms, const float* x,
                               uint32_t* key, uint32_t* perm, uint32_t* start, uint32_t* count, int* status,
                               void* stream);

void fmm_destroy(fmm_handle* h);
const char* fmm_error_string(fmm_status s);
/* Detail of the last CUDA failure reported by this thread (the failing call and CUDA's
 * message); an empty string when none has been recorded. */
const char* fmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FMMCPH_H */
