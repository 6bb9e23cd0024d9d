/*
 * lo_afqmc.h -- C ABI of the B300 (sm_103a) LO-AFQMC local-energy library.
 *
 * The library evaluates, for a batch of walkers, the phaseless-AFQMC local
 * energy  E = <Phi_T|H|phi> / <Phi_T|phi>  of a single-determinant trial
 * (Weber et al., arXiv 2202.00832, Sec. 2.1.1, generalized Wick form eq.
 * 2e_general), through the half-rotated Cholesky vectors (Sec. 2.2, eq.
 * 2e_HRchol_RCAS) -- the "full" path -- or with the exchange taken from the
 * SVD-truncated localized-orbital pair blocks (Sec. 3.1, eqs. 2e_HR_RCAS_LO
 * and 2e_HR_RCAS) -- the "LO" path.
 *
 * Conventions for every entry point
 *   - Matrices are row-major, FP64 real or complex128 (re, im interleaved).
 *   - M = basis size, X = number of Cholesky vectors, n_alpha / n_beta =
 *     occupied orbitals per spin, W = walkers in a call.
 *   - A closed shell (n_alpha == n_beta and no trial_b) uses one restricted
 *     determinant per walker for both spins.
 *   - "device" buffers are CUDA device pointers on the context's device;
 *     "host" buffers are ordinary or pinned host memory.  Entry points that
 *     accept either say so and detect the kind with cudaPointerGetAttributes.
 *   - All GPU work is queued on the context's stream; calls return after the
 *     results they write to host memory are complete.  Device outputs are
 *     complete when the stream reaches the end of the call.
 *   - Every call returns a loaf_status.  No call aborts, exits or traps on
 *     the device; loaf_last_error() describes the most recent failure.
 */
#ifndef LO_AFQMC_H
#define LO_AFQMC_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct loaf_ctx loaf_ctx; /* opaque; owns every device buffer it allocates */

typedef enum {
    LOAF_OK = 0,
    LOAF_ERR_ARG = 1,         /* null pointer or out-of-range scalar argument */
    LOAF_ERR_SHAPE = 2,       /* sizes inconsistent or beyond supported limits */
    LOAF_ERR_CUDA = 3,        /* a CUDA runtime / library call failed */
    LOAF_ERR_OOM = 4,         /* device allocation failed */
    LOAF_ERR_SINGULAR = 5,    /* at least one walker overlap is singular */
    LOAF_ERR_NOT_READY = 6,   /* required setup call has not been made */
    LOAF_ERR_TIMEOUT = 7,     /* a bounded device wait gave up */
    LOAF_ERR_NAN = 8,         /* non-finite input or result */
    LOAF_ERR_UNSUPPORTED = 9  /* valid request this library does not provide */
} loaf_status;

enum { LOAF_MODE_FULL = 0, LOAF_MODE_LO = 1, LOAF_MODE_LO_JK = 2 };

/*
 * Arithmetic of the contractions (the final per-walker accumulation is FP64
 * in every mode):
 *   LOAF_PREC_FP64   every step in FP64 (CUDA cores).
 *   LOAF_PREC_FP16X3 Coulomb and LO-exchange contractions on the tcgen05
 *                    tensor cores: operands split into FP16 hi + lo parts
 *                    (power-of-two scaled), three products hi*hi + hi*lo +
 *                    lo*hi accumulated in FP32, applied to Theta - Phi_T
 *                    (the walker-independent trial part stays FP64).  In the
 *                    LO modes the overlap S and Theta = phi S^-1 are exact
 *                    products of 7-bit digit slices on the tensor cores, and
 *                    S^-1 and log det S come from a double-float (2 x FP32,
 *                    about 48 significant bits) Gauss-Jordan elimination.
 *   LOAF_PREC_BF16X3 the same with BF16 hi + lo parts.
 *   LOAF_PREC_FP16X3_F64INV  LOAF_PREC_FP16X3 with S^-1 and log det S from a
 *                    Gauss-Jordan elimination in FP64 (the overlap inversion
 *                    and log-determinant kept in FP64 end to end).
 *   LOAF_PREC_TF32   the Coulomb and LO-exchange contractions as one TF32
 *                    product each (kind::tf32, FP32 accumulation) on the same
 *                    Theta - Phi_T; overlap, inverse and Theta as for FP16X3;
 *                    every pair through its dense truncated block.  Mode LO
 *                    only (walkers_energy, walkers_pair_exchange);
 *                    LOAF_ERR_UNSUPPORTED elsewhere.  About 11 significant bits
 *                    per operand: a reference point for the split products,
 *                    not a production precision.
 */
enum { LOAF_PREC_FP64 = 0, LOAF_PREC_FP16X3 = 1, LOAF_PREC_BF16X3 = 2, LOAF_PREC_FP16X3_F64INV = 3,
       LOAF_PREC_TF32 = 4 };

/* Per-walker status codes written to walker_status[] */
enum { LOAF_WALKER_OK = 0, LOAF_WALKER_SINGULAR = 1, LOAF_WALKER_NAN = 2 };

/* Supported limits of this library. */
#define LOAF_MAX_NOCC 96      /* occupied orbitals per spin (LU held in shared memory) */
#define LOAF_MAX_BASIS 1536

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL: the context creates its own non-blocking stream).  On success *ctx
 * owns no device memory yet. */
loaf_status loaf_create(loaf_ctx **ctx, int device, void *cuda_stream);

/* Free every device buffer and library handle the context owns. NULL is a no-op. */
loaf_status loaf_destroy(loaf_ctx *ctx);

/* Static description of a status code. */
const char *loaf_status_str(loaf_status s);

/* Message for the last failing call on this context (never NULL). */
const char *loaf_last_error(const loaf_ctx *ctx);

/*
 * ao_load_cholesky -- load the Hamiltonian and the trial; half-rotate.
 *
 * Sec. 2.1 (H = sum h_pq c+_p c_q + 1/2 sum V_pqrs ..., V_pqrs = sum_g
 * L^g_pr L^g_qs) and Sec. 2.2 (Lbar^g_ir = sum_p L^g_rp Phi_T,pi, computed
 * once before propagation).
 *   h        M x M, symmetric one-body matrix
 *   L        X x M x M, each slice symmetric (Cholesky vectors)
 *   trial_a  M x n_alpha, orthonormal columns (real trial determinant)
 *   trial_b  M x n_beta, or NULL for a closed shell (n_beta == n_alpha)
 *   e0       constant added to every energy
 *   inputs_on_device  0: the four arrays are host memory; 1: device memory.
 * The arrays are copied; the caller keeps ownership.  Re-calling replaces the
 * system and drops any LO compression.  Errors: LOAF_ERR_SHAPE for M, X,
 * n_alpha, n_beta outside (1..LOAF_MAX_BASIS, 1.., 1..min(M, LOAF_MAX_NOCC));
 * LOAF_ERR_OOM when the device cannot hold L.
 */
loaf_status ao_load_cholesky(loaf_ctx *ctx, int M, int X, const double *h, const double *L,
                             int n_alpha, int n_beta, const double *trial_a,
                             const double *trial_b, double e0, int inputs_on_device);

/*
 * lo_localize_compress -- Foster-Boys localization and pair compression.
 *
 * Sec. 4 (Foster-Boys localization of the occupied orbitals) and Sec. 3.1.1:
 * for every pair i <= j of localized orbitals the M x M block
 * Y^[ij]_rs = sum_g Lbar^g_ir Lbar^g_js is factorised by SVD and truncated,
 * keeping the singular values s >= t_svd (absolute, Hartree):
 * Y^[ij] ~= Ubar Vbar with Ubar = U sqrt(s), Vbar = sqrt(s) V^T.
 *   t_svd     >= 0; 0 keeps every singular value (exact)
 *   r_ops     n_ops x M x M symmetric position-operator matrices in the
 *             orthonormal basis (host memory), e.g. diag(x), diag(y), diag(z)
 *   localize  1: Boys-localize first; 0: keep the canonical trial orbitals
 *   compression_pct  out (host, may be NULL): (M - <M_SVD>)/M*100 over all
 *             pairs and spins (Sec. 4)
 *   m_svd_per_pair   out (host, may be NULL): kept rank of every pair, spin
 *             alpha pairs (0,0),(0,1)..(0,N-1),(1,1).. then spin beta
 * May be re-called with another t_svd or localize; the SVDs are recomputed.
 * Errors: LOAF_ERR_NOT_READY before ao_load_cholesky.
 */
loaf_status lo_localize_compress(loaf_ctx *ctx, double t_svd, const double *r_ops, int n_ops,
                                 int localize, double *compression_pct, int *m_svd_per_pair);

/*
 * walkers_energy -- local energies of W walkers (the hot path).
 *
 * For each walker: S = Phi_T^T phi (per spin), partial-pivot LU of S,
 * log det S, Theta = phi S^-1 (eq. Q), then E = e0 + E1 + E_J - E_K with the
 * one-body E1 = sum_sigma sum_ir hbar_ir Theta_ri, the Coulomb
 * E_J = 1/2 sum_g (sum_sigma tr Lbar^sigma_g Theta^sigma)^2 and the exchange
 * E_K = 1/2 sum_sigma sum_g tr(T T), T = Lbar^sigma_g Theta^sigma (mode FULL,
 * eq. 2e_HRchol_RCAS) or E_K = 1/2 sum_sigma sum_ij e_ij with
 * e_ij = (Ubar^[ij]T Theta_j).(Vbar^[ij] Theta_i) (mode LO, eq. 2e_HR_RCAS_LO).
 *   W          >= 1 walkers
 *   phi        W x M x Ntot complex128, Ntot = n_alpha (closed shell) or
 *              n_alpha + n_beta (alpha columns first); host or device
 *   mode       LOAF_MODE_FULL, LOAF_MODE_LO (LO needs lo_localize_compress), or
 *              LOAF_MODE_LO_JK: LO exchange and the Coulomb from the same
 *              compressed pair factors, E_J = 2 sum_ij (Ubar^[ij]T Theta_i).
 *              (Vbar^[ij] Theta_j) (eq. 2e_HR_RCAS, the 4 Q_ri Q_sj term; closed
 *              shells only, LOAF_ERR_UNSUPPORTED otherwise)
 *   precision  LOAF_PREC_*; the full mode supports FP64 and FP16X3/BF16X3
 *              (Coulomb on tensor cores, exchange FP64)
 *   e_out      W complex128 energies (host or device)
 *   logdet_out W complex128 log <Phi_T|phi> = sum_sigma log det S^sigma, or NULL
 *   walker_status  W ints (host or device), or NULL
 * A singular overlap marks that walker LOAF_WALKER_SINGULAR, writes NaN to
 * its energy and makes the call return LOAF_ERR_SINGULAR after finishing the
 * others.  Workspace grows to the largest W seen and is kept by the context.
 * A host phi of W >= 512 walkers is uploaded in chunks while the previous
 * chunk computes; the call returns when every output has been written.
 */
loaf_status walkers_energy(loaf_ctx *ctx, int W, const void *phi, int mode, int precision,
                           void *e_out, void *logdet_out, int *walker_status);

/*
 * walkers_energy_submit / walkers_energy_wait -- walkers_energy as a stream
 * of calls.  The same computation and outputs as walkers_energy (eq. Q and
 * eq. 2e_HR_RCAS_LO for mode LO; the same kernels, so results identical to a
 * walkers_energy call on the same W device-resident walkers), but submit
 * returns once the work is queued: the upload of one call's walkers (host
 * phi, two copies on two copy streams) runs while the previous call computes.
 * Two calls alternate between two device copies of the walkers owned by the
 * context; submitting a third first waits for the first.
 *   arguments as walkers_energy; host buffers must stay valid and unread
 *   until walkers_energy_wait returns, and must be page-locked (pinned) for
 *   the copies to overlap (pageable buffers work but serialise the call).
 *   A change of (W, mode, precision) between submitted calls first waits for
 *   those in flight (the workspace is sized for one shape at a time), and so
 *   do ao_load_cholesky, lo_localize_compress, loaf_set_tiles (when the shapes
 *   change), pair_screen_train, pair_screen_set and walkers_energy_multi: a
 *   queued call computes with the operands it was queued with.
 * Errors: argument errors as walkers_energy, at submit.  Walker failures and
 * pipeline timeouts of the submitted calls are reported by walkers_energy_wait
 * (LOAF_ERR_SINGULAR / LOAF_ERR_NAN / LOAF_ERR_TIMEOUT, the worst over the
 * calls since the last wait); each call's walker_status marks its walkers.
 * walkers_energy_wait returns when every submitted call's outputs are written.
 */
loaf_status walkers_energy_submit(loaf_ctx *ctx, int W, const void *phi, int mode, int precision,
                                  void *e_out, void *logdet_out, int *walker_status);
loaf_status walkers_energy_wait(loaf_ctx *ctx);

/*
 * loaf_set_tiles / loaf_get_tiles -- tile shapes of the tensor-core kernels of
 * one context (the paper has no counterpart: its batched contractions of
 * Sec. 4.4 leave the tiling to the GEMM library).
 *   lo_chunk_cap   the largest chunk of a pair's rows (kept ranks, or rows of a
 *                  dense truncated block) one LO unit takes as the MMA's N
 *                  dimension; a pair's rows are cut into balanced chunks of at
 *                  most this many (a multiple of 16 each).  A multiple of 32 in
 *                  [64, 256]; default 256.
 *   coulomb_split  how many parts the Coulomb contraction over (orbital, basis)
 *                  is split into across CTA pairs; 0 (default) = the rule that
 *                  fills the last round of the persistent grid to >= 90 %.
 * The shapes change only the order of the sums (the split also moves the
 * boundaries of the 128-term FP32 accumulation chains), not the method.  A new
 * chunk cap rebuilds the LO operands on the next call.  walkers_energy_multi
 * with autotune = 1 sets both per context by timing candidates; loaf_get_tiles
 * reads the shapes in use.  Errors: LOAF_ERR_ARG for a NULL context or a value
 * out of range (the shapes are left unchanged).
 */
loaf_status loaf_set_tiles(loaf_ctx *ctx, int lo_chunk_cap, int coulomb_split);
loaf_status loaf_get_tiles(const loaf_ctx *ctx, int *lo_chunk_cap, int *coulomb_split);

/*
 * walkers_energy_multi -- local energies of several systems in one launch.
 *
 * The walkers_energy computation (mode LO, precision FP16X3 or BF16X3) for n
 * loaded contexts (for example molecules of different sizes), each with its
 * own batch, recorded once as a single CUDA graph whose branches run side by
 * side and replayed on later calls with the same signature (contexts, sizes,
 * buffers, loaded trial, screen and tile shapes).  With autotune = 1 the first
 * call also chooses, for each system with the GPU to itself, its tile shapes
 * (loaf_set_tiles: the LO chunk cap among 256, 192 and 128, then the Coulomb
 * split among the rule's, half and twice it) by timing eager calls, and keeps
 * them in the context; then how many SMs the persistent kernels of each
 * system may fill in the graph (all of them, or shares proportional to each
 * system's LO work) by timing the candidate graphs; sm_caps reports that
 * choice and loaf_get_tiles the shapes.
 *   ctxs          n distinct contexts on the same device, each after
 *                 lo_localize_compress
 *   W             n batch sizes (>= 1)
 *   phi           n device arrays, W[k] x M_k x Ntot_k complex128
 *   e_out         n device arrays of W[k] complex128
 *   logdet_out    n device arrays of W[k] complex128, or NULL (array or entries)
 *   walker_status n device arrays of W[k] ints, or NULL (array or entries)
 *   sm_caps       out (host, may be NULL): n SM budgets used (0 = all)
 * Device buffers only (the graph keeps their addresses).  Errors as for
 * walkers_energy; LOAF_ERR_ARG for host buffers or repeated contexts,
 * LOAF_ERR_UNSUPPORTED for another mode or precision.  The call returns when
 * every system's outputs are written.
 */
loaf_status walkers_energy_multi(loaf_ctx *const *ctxs, int n, const int *W, const void *const *phi,
                                 int mode, int precision, void *const *e_out,
                                 void *const *logdet_out, int *const *walker_status, int autotune,
                                 int *sm_caps);

/*
 * walkers_force_bias -- the mixed estimate of every Cholesky vector,
 * <L_g>_w = sum_sigma tr(Lbar^sigma_g Theta^sigma) (g < X), the quantity the
 * importance-sampled propagation shifts the auxiliary fields by (the force
 * bias -sqrt(dtau) <L_g>, Sec. 2.1; mean-field subtraction is the caller's).
 * It is the Coulomb vector of walkers_energy, formed by the same kernels.
 *   W, phi         as for walkers_energy (host or device)
 *   precision      LOAF_PREC_FP64 or the split precisions
 *   lbar_out       W x X complex128 (walker-major), host or device
 *   logdet_out, walker_status  as for walkers_energy (may be NULL)
 * Needs ao_load_cholesky only.  Errors as for walkers_energy.
 */
loaf_status walkers_force_bias(loaf_ctx *ctx, int W, const void *phi, int precision, void *lbar_out,
                               void *logdet_out, int *walker_status);

/*
 * walkers_propagator -- the one-body operator of each walker's propagator,
 * V_w = sum_g x_wg L_g (M x M; the B = sum_alpha x_alpha L_alpha formation of
 * the propagation step, Sec. 2.1 and Sec. 5), for fields x that already hold
 * sqrt(dtau) and the force-bias shift.
 *   W          >= 1 walkers
 *   x          W x X complex128 fields (walker-major), host or device
 *   precision  LOAF_PREC_FP64 (cuBLAS DGEMMs) or a split precision (one
 *              tensor-core contraction over g with 16-bit hi + lo tiles)
 *   v_out      W x M x M complex128 (v_out[w][p][q]), host or device
 * Needs ao_load_cholesky only; L must be kept by the context (it is).  The
 * split-precision operand tiles of L are built on the first call.
 * Errors: LOAF_ERR_NOT_READY, LOAF_ERR_ARG, LOAF_ERR_OOM, LOAF_ERR_TIMEOUT.
 */
loaf_status walkers_propagator(loaf_ctx *ctx, int W, const void *x, int precision, void *v_out);

/*
 * walkers_energy_cas -- mixed-estimate local energy with a multi-determinant
 * (CAS) trial sum_d c_d |Phi_d>, through Sherman-Morrison-Woodbury updates of
 * the reference determinant (Sec. 3.1.2: eqs. Q_SMW_reg, Q_SMW, BigQ and
 * 2e_HR_RCAS).  FP64 (the projections onto the factor rows in double-float,
 * about 48 significant bits).  The context holds the CAS orbitals as its trial:
 * ao_load_cholesky with a closed shell of n_alpha = n_beta = n_cas orbitals
 * (inactive orbitals first, localized as the caller wants them), then
 * lo_localize_compress(localize = 0) for the factors of every CAS orbital pair.
 * Every determinant is closed shell and occupies N of the CAS orbitals.
 *   W, N       walkers; occupied orbitals per spin (1 <= N <= min(64, n_cas))
 *   phi        W x M x N complex128 walkers (both spins alike), host or device
 *   n_det      number of determinants (>= 1)
 *   dets       n_det x N int32 (host): the CAS orbital in each slot; dets[0] is
 *              the reference, and every other determinant keeps the reference's
 *              orbital in all but at most 8 slots
 *   coeffs     n_det doubles (host): c_d
 *   e_out      W complex128: sum_d c_d <Phi_d|phi> E_d / sum_d c_d <Phi_d|phi>
 *   logov_out  W complex128 or NULL: log sum_d c_d <Phi_d|phi> (both spins)
 *   walker_status  W ints (LOAF_WALKER_*) or NULL
 * A determinant whose overlap with a walker is exactly zero gets weight 0.
 * Workspace on the device grows with W (X + 1) n_cas C and W (sum of kept
 * ranks) C complex values, C = 1 + the number of slots some determinant changes.  Errors: LOAF_ERR_NOT_READY without
 * lo_localize_compress or for an open shell; LOAF_ERR_SHAPE for N or an
 * excitation rank beyond the limits; LOAF_ERR_ARG for an orbital index outside
 * 0..n_cas-1 or repeated within a determinant; LOAF_ERR_SINGULAR /
 * LOAF_ERR_NAN when a reference overlap is singular / not finite (the other
 * walkers are still evaluated).
 */
loaf_status walkers_energy_cas(loaf_ctx *ctx, int W, int N, const void *phi, int n_det, const int *dets,
                               const double *coeffs, void *e_out, void *logov_out, int *walker_status);

/*
 * walkers_theta -- the first stage alone: Theta = phi (Phi_T^T phi)^-1 and
 * log det, per spin (eq. Q).  theta_out: W x Ntot x M complex128 (orbital-
 * major: theta_out[w][i][r] = Theta_ri), logdet_out: W complex128.  The
 * trial is the canonical one, or the localized one after
 * lo_localize_compress(localize=1) (Theta changes by that rotation).
 * Buffers host or device.
 */
loaf_status walkers_theta(loaf_ctx *ctx, int W, const void *phi, void *theta_out,
                          void *logdet_out, int *walker_status);

/*
 * walkers_pair_exchange -- the LO pair values e^sigma_ij(w) of eq. 2e_HR_RCAS
 * (exchange part), unweighted, for every stored pair i <= j.
 *   e_pairs_out  n_pairs_total x W complex128 (pair-major; pair order as in
 *                m_svd_per_pair), host or device
 */
loaf_status walkers_pair_exchange(loaf_ctx *ctx, int W, const void *phi, int precision,
                                  void *e_pairs_out);

/* Number of stored pairs over all spins (0 before lo_localize_compress). */
int loaf_num_pairs(const loaf_ctx *ctx);

/*
 * lo_get_localized_trial -- copy the trial orbitals the LO factors were built
 * from (M x n_sigma, host) for spin 0 (alpha) or 1 (beta).
 */
loaf_status lo_get_localized_trial(const loaf_ctx *ctx, int spin, double *out);

/*
 * Learned pair screen.  The paper's conclusions (Sec. 5) propose screening
 * electron pairs and keeping only those that contribute meaningfully; they
 * give no algorithm.  Here a network 8 -> 64 -> 64 -> 1 (tanh hidden layers,
 * FP16 weights and activations, FP32 accumulation) predicts log10 of the
 * largest |e_ij| of each pair [ij] from eight walker-independent descriptors
 * (centroid distance d, 1/(1+d), spread sum and difference of the two
 * localized orbitals, log s_1, log s_2, M_SVD/M, log |Y^[ij]|_F); pairs
 * predicted below a cutoff are left out of the LO exchange (their trial part
 * e0 included).  The unscreened evaluation stays available.
 *
 * pair_screen_train: computes the training labels with the FP16X3 LO path on
 *   W_train walkers (phi as in walkers_energy, host or device), standardises
 *   descriptors and labels, and runs `epochs` full-batch Adam steps (beta1 0.9,
 *   beta2 0.999, eps 1e-8, learning rate lr) from init_params (host,
 *   loaf_screen_num_params() floats in the order W1[64][8], b1[64], W2[64][64],
 *   b2[64], W3[64], b3).  loss_history (host, `epochs` floats, may be NULL)
 *   receives the mean squared error before each step.  Clears any screen.
 * pair_screen_set: cutoff_ha >= 0 keeps pairs with predicted |e_ij| >= cutoff;
 *   cutoff_ha < 0 removes the screen.  kept_pairs (may be NULL) gets the count.
 * pair_screen_query: copies (each may be NULL) the trained parameters, the
 *   8 descriptors of every pair (double, pair-major), the predicted and the
 *   label log10 |e_ij|, and the keep mask (1 = evaluated).
 * mlp_loss_grad: the network's mean squared error and its gradient with
 *   respect to the parameters on n standardised samples x (n x 8) and
 *   targets t (host arrays), on CUDA device `device` -- the kernels training
 *   uses, exposed for gradient checks.
 */
int loaf_screen_num_params(void);
loaf_status pair_screen_train(loaf_ctx *ctx, int W_train, const void *phi, int epochs, float lr,
                              const float *init_params, float *loss_history);
loaf_status pair_screen_set(loaf_ctx *ctx, double cutoff_ha, int *kept_pairs);
loaf_status pair_screen_query(const loaf_ctx *ctx, float *params_out, double *features_out,
                              double *pred_log10_out, double *target_log10_out,
                              unsigned char *keep_out);
loaf_status mlp_loss_grad(int device, int n, const float *x, const float *t, const float *params,
                          float *loss_out, float *grad_out);

/*
 * walkers_theta_noalloc -- walkers_theta for callers that may not allocate
 * device memory while they run: code that owns a fixed memory budget (an
 * allocator that hands out one arena up front, a job that must not grow its
 * footprint once it is running), or code that runs while allocation is off
 * limits.  The paper has no counterpart; it is a deployment variant of the
 * first stage only.
 *
 * Same result as walkers_theta (Theta = phi (Phi_T^T phi)^-1 per spin and
 * log <Phi_T|phi>), but every buffer is the caller's and on the device, and
 * the kernel's scratch lives in one fixed 32 MiB array compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  No cudaMalloc, cudaFree or allocating library routine is called.
 *   phi            device, W x M x Ntot complex128
 *   theta_out      device, W x Ntot x M complex128 (orbital-major)
 *   logdet_out     device, W complex128, or NULL
 *   walker_status  device, W ints, or NULL (singular walkers are reported
 *                  here only; the call itself returns LOAF_OK)
 * Limits: 1 <= W <= 4096 and W * Ntot * M <= 2,086,912; larger requests are
 * rejected with LOAF_ERR_SHAPE before any work is queued.
 * The call is asynchronous on the context stream.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other contexts on the
 * same device, other threads) race on it and must be serialised by the caller.
 */
loaf_status walkers_theta_noalloc(loaf_ctx *ctx, int W, const void *phi, void *theta_out,
                                  void *logdet_out, int *walker_status);

/*
 * loaf_test_withhold_stage -- failure-path test hook (the paper has no
 * counterpart).  The next n launches of the tensor-core LO exchange kernel on
 * this context leave the first pipeline stage of one CTA pair unfilled: no
 * copy is issued and no arrival is made, so that pair's bounded mbarrier waits
 * run out after their limit (1 s of %globaltimer), every role of both CTAs
 * leaves its loop, copies already issued are waited for (bounded), TMEM is
 * freed, and the call that launched it returns LOAF_ERR_TIMEOUT.  Nothing
 * faults or hangs; the context stays usable.  n = 0 (the default) turns it
 * off.  Errors: LOAF_ERR_ARG for a NULL context or n < 0.
 */
loaf_status loaf_test_withhold_stage(loaf_ctx *ctx, int n);

/*
 * Stage timers.  loaf_profile(ctx, 1) resets and enables CUDA-event timers
 * around every stage a call launches (events on the context stream, read
 * after the call's final synchronisation); loaf_profile(ctx, 0) disables
 * them.  loaf_profile_get returns, for stage idx < loaf_profile_count(ctx),
 * its name (owned by the context, valid until the next loaf_profile call),
 * the summed elapsed time in ms, the number of timed calls and the number of
 * kernel launches those calls made.  Timers add two event records per stage.
 */
loaf_status loaf_profile(loaf_ctx *ctx, int enable);
int loaf_profile_count(const loaf_ctx *ctx);
loaf_status loaf_profile_get(const loaf_ctx *ctx, int idx, const char **name, double *total_ms,
                             long *calls, long *launches);

#ifdef __cplusplus
}
#endif
#endif /* LO_AFQMC_H */
