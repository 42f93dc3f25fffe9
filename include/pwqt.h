/*
 * pwqt.h -- C ABI of libpwqt: the per-energy open-boundary solve of the
 * partition-of-unity Bloch-wave method (Van de Put, Fischetti, Vandenberghe,
 * arXiv:1903.00548) on one GB300 GPU.
 *
 * Conventions (all entry points):
 *  - Every function returns an int status: PWQT_OK (0) or a negative PWQT_ERR_*
 *    code; pwqt_last_error(ctx) returns a message for the last failure.
 *  - Complex numbers are interleaved double[2] (re, im).  Matrices are row-major.
 *  - Host arrays are owned by the caller and only read or written during the
 *    call; the library never keeps a pointer to them and never returns memory
 *    that the caller must free.
 *  - Device state (intrinsic blocks, per-node extrinsic blocks, the cache of
 *    contact self-energies, factor panels) is owned by the opaque context and
 *    released by pwqt_destroy.
 *  - Units: eV for energies and potentials, nm for lengths.
 *  - A context is thread-compatible, not thread-safe: use one host thread per
 *    context.  Every computation runs in the library's CUDA kernels (and the
 *    cuSOLVER/cuBLAS calls named below) on the context's device; there is no
 *    CPU fallback: without a usable CUDA device pwqt_create fails.
 */
#ifndef PWQT_H
#define PWQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pwqt_ctx pwqt_ctx;

/* return codes */
#define PWQT_OK                   0
#define PWQT_ERR_INVALID_ARG     -1   /* a pointer is NULL, a size is out of range */
#define PWQT_ERR_BASIS_TOO_SMALL -2   /* fewer plane waves than requested bands    */
#define PWQT_ERR_OOM             -3   /* device allocation or HBM budget exceeded  */
#define PWQT_ERR_CUDA            -4   /* a CUDA runtime / library call failed      */
#define PWQT_ERR_STATE           -5   /* call order violated (e.g. no basis yet)   */
#define PWQT_ERR_NO_DEVICE       -6   /* no CUDA device / driver                   */
#define PWQT_ERR_TIMEOUT         -7   /* a bounded wait gave up (device-side wait,
                                         or pwqt_server_wait before completion);
                                         if a tensor-core kernel could not drain its
                                         MMAs it keeps their tensor memory and the
                                         device is unfit for more tensor-core work */
#define PWQT_ERR_BUSY            -8   /* the server's request queue is full        */

/* per-result status bits (pwqt_solve `status` output) */
#define PWQT_ST_OK               0
#define PWQT_ST_SINGULAR_PIVOT   1    /* a pivot of a node block was exactly zero   */
#define PWQT_ST_MODE_COUNT       2    /* out-flow mode count != n at a contact     */
#define PWQT_ST_IR_NO_CONVERGE   4    /* refinement stopped above its tolerance    */
#define PWQT_ST_DEGENERATE       8    /* degenerate traveling modes at a contact   */
#define PWQT_ST_NEAR_UNIT        16   /* an evanescent |lambda| within 1e-3 of 1   */

/* precision of the block sweep */
#define PWQT_FP64                0    /* complex128 throughout                     */
#define PWQT_MIXED               1    /* complex64 factorisation on the tensor
                                         cores (3xTF32 products, FP32 accumulate)
                                         + refinement with FP64-accurate residuals
                                         (see pwqt_set_residual)                   */
#define PWQT_FP32                2    /* the complex64 factorisation alone (no
                                         refinement; resid reports its residual)   */

typedef struct {
    int    device;             /* CUDA device ordinal                              */
    size_t hbm_budget_bytes;   /* 0: use 90 % of the free device memory            */
    double ir_tol;             /* mixed path: stop when ||B - A c|| <= ir_tol ||B||
                                  (max over columns); 0 -> 1e-10.  A residual that
                                  stops falling above it ends the refinement with
                                  PWQT_ST_IR_NO_CONVERGE                            */
    int    ir_max_iters;       /* mixed path refinement limit; 0 -> 40              */
    int    batch;              /* energies per sweep launch; 0 -> from the budget   */
} pwqt_opts;

/* One periodic supercell (paper Sec. 2.1, Fig. structure). */
typedef struct {
    int           dim;        /* 1: chain along z; 2: ribbon in the x-z plane      */
    double        Lz;         /* supercell length along transport (nm)             */
    double        Lx;         /* transverse supercell width (nm); 1 for dim == 1    */
    int           n_atoms;
    const double* atoms;      /* n_atoms x 2 (x, z) positions, nm                  */
    double        omega0;     /* reference volume per atom of the form factor      */
} pwqt_cell;

/* Local empirical pseudopotential v(q) = v0 exp(-q^2 / (2 sigma^2))
   (Sec. 2.1, Eq. local_epp; Sec. 1: V(q) a continuous function of q). */
typedef struct {
    double v0;                /* eV    */
    double sigma;             /* nm^-1 */
} pwqt_formfactor;

/* Create a context on opts->device (NULL: defaults, device 0).
   Errors: PWQT_ERR_NO_DEVICE, PWQT_ERR_CUDA, PWQT_ERR_INVALID_ARG (out NULL). */
int pwqt_create(pwqt_ctx** out, const pwqt_opts* opts);

/* Release all device state of the context.  NULL is accepted. */
int pwqt_destroy(pwqt_ctx* ctx);

/* Message of the last failing call on this context (static storage of ctx). */
const char* pwqt_last_error(const pwqt_ctx* ctx);

/*
 * Intrinsic blocks from the pseudopotential (Sec. 2.2-2.3, App. A).
 * Builds the plane-wave EPM Hamiltonian H_GG' = hbar^2/2m |k+G|^2 delta +
 * V_{G-G'} (plane waves |k+G| <= gcut; V_G = (omega0/Omega) v(|G|) sum_a
 * e^{-iG.R_a}, V_0 = 0) at k = 0 and k = pi/Lz, keeps the n_bands lowest Bloch
 * waves of each (n = 2 n_bands enhancement functions per node, Eq.
 * wavef_expansion), and forms the element integrals M, H^c = (eps+eps')/2 M +
 * T + P (Eq. hc_matel_herm) and the extrinsic weights W (Sec. 2.3) in closed
 * form.  Resets all systems and the self-energy cache.
 *   n_out: receives n.
 * Errors: PWQT_ERR_BASIS_TOO_SMALL if a k-point has fewer than n_bands plane
 * waves; PWQT_ERR_INVALID_ARG; PWQT_ERR_CUDA (cuSOLVER Hermitian eigensolver).
 */
int pwqt_assemble_intrinsic(pwqt_ctx* ctx, const pwqt_cell* cell, const pwqt_formfactor* ff,
                            double gcut, int n_bands, int* n_out);

/*
 * Same as pwqt_assemble_intrinsic, but with caller-supplied Bloch waves
 * (Sec. 2.2: "Bloch-wave solutions ... obtained ... using the appropriate
 * plane-wave basis").  Group g = 0 is k = 0, g = 1 is k = pi/Lz.
 *   eps   : 2*n_bands band energies, group 0 first.
 *   n_pw  : 2 counts of plane waves.
 *   mx, mz: n_pw[0] + n_pw[1] integer plane-wave indices, G = (2 pi mx/Lx, 2 pi mz/Lz).
 *   coef  : complex, group 0 then group 1, each n_pw[g] x n_bands row-major,
 *           normalised to sum_G |c|^2 = 1 per band.
 */
int pwqt_set_enhancement(pwqt_ctx* ctx, const pwqt_cell* cell, int n_bands, const double* eps,
                         const int* n_pw, const int* mx, const int* mz, const double* coef,
                         int* n_out);

/*
 * Copies of the intrinsic node blocks (Eq. infinite_system), each n x n complex:
 * H0 = H_ii, H1 = H_{i,i+1}, M0 = M_ii, M1 = M_{i,i+1}, and W (6 blocks:
 * W^l_ll, W^l_lr, W^l_rr, W^r_ll, W^r_lr, W^r_rr).  Any pointer may be NULL.
 */
int pwqt_get_blocks(pwqt_ctx* ctx, double* H0, double* H1, double* M0, double* M1, double* W);

/*
 * Extrinsic potential of system `sys` (0 <= sys < 64): U_nodes[i] is the
 * potential energy at node i+1 (i < n_nodes), interpolated by the hats,
 * V_e(z) = sum_j U_j f_j(z) (Sec. 2.3 V^e elements); the leads are flat at
 * U_nodes[0] and U_nodes[n_nodes-1].  Builds the per-node blocks H_ii + V_ii
 * and H_{i,i+1} + V_{i,i+1} on the device.  n_nodes >= 2.
 */
int pwqt_set_extrinsic(pwqt_ctx* ctx, int sys, int n_nodes, const double* U_nodes);

/*
 * Solve [E M - H - Sigma] c = B (Eq. qtbm_system) for every injected mode at
 * each of the n_E energies of system `sys`, and reduce to observables.
 * Self-energies (Sec. 3.1: complex bands of the flat leads from the symmetric
 * linearisation, Eq. linearized_eigenvalue_symmetric; velocities, Eq.
 * hellmann-feynman; normalisation, Eq. normalization) come from the context's
 * cache, keyed by E - U_lead, and are computed on a miss (cuSOLVER non-Hermitian
 * eigensolver + the library's kernels, FP64).
 * Outputs (host, caller-owned, any may be NULL):
 *   T      [n_E]        sum over source-injected modes of T_gamma (Eq. transmission)
 *   R      [n_E]        sum of the source reflection coefficients
 *   T_ds   [n_E]        drain -> source transmission
 *   n_open [2*n_E]      injected traveling modes (source, drain)
 *   node_n [n_E*N*2]    node density per contact, g_gamma sum_alpha |c|^2 (Sec. 3.3)
 *   resid  [n_E]        final max-column ||B - A c|| / ||B|| (FP64 residual)
 *   iters  [n_E]        refinement iterations (0 on the FP64 path)
 *   status [n_E]        PWQT_ST_* bits
 */
int pwqt_solve(pwqt_ctx* ctx, int sys, int n_E, const double* E, int precision,
               double* T, double* R, double* T_ds, int* n_open, double* node_n,
               double* resid, int* iters, int* status);

/*
 * pwqt_solve for several systems (e.g. bias points of one device, Sec. 4: the
 * solve repeated for every applied potential) at the same n_E energies: results
 * are system-major, entry s * n_E + e for system sys_ids[s]; node_n holds
 * n_E * N_s * 2 values per system, systems back to back in the order given.
 * When the systems share one node count (and, for PWQT_MIXED / PWQT_FP32, the
 * sliced residual is selected) every (system, energy) pair runs in the same
 * batched launches -- each job carries its own system's node blocks, and the
 * self-energy cache serves every bias point whose leads sit at the same energy;
 * otherwise system by system.  Errors: as pwqt_solve (in the system-by-system
 * case nothing is written past the first failing system's block).
 */
int pwqt_solve_multi(pwqt_ctx* ctx, int n_sys, const int* sys_ids, int n_E, const double* E, int precision,
                     double* T, double* R, double* T_ds, int* n_open, double* node_n,
                     double* resid, int* iters, int* status);

/*
 * pwqt_solve on device buffers: E (n_E doubles) and every output are device
 * pointers (any output may be NULL), the work is ordered on `stream`
 * (a cudaStream_t, NULL = the legacy default stream) and the call returns once
 * it is enqueued and the self-energy cache holds every needed entry (cache
 * misses are computed synchronously first).  The buffers must stay valid until
 * the stream reaches the end of the work.
 */
int pwqt_solve_dev(pwqt_ctx* ctx, int sys, int n_E, const double* E_host, int precision,
                   double* T, double* R, double* T_ds, int* n_open, double* node_n,
                   double* resid, int* iters, int* status, void* stream);

/*
 * Pre-fill the self-energy cache for energies E - U_lead of system `sys`
 * (both leads), so that a later pwqt_solve runs with resident self-energies.
 */
int pwqt_prepare_leads(pwqt_ctx* ctx, int sys, int n_E, const double* E);

/* Number of cached contact entries and the device bytes they hold. */
int pwqt_cache_info(pwqt_ctx* ctx, int* entries, size_t* bytes);

/*
 * Band reconstruction (Sec. 5.1): eigenvalues of H(k') c = E M(k') c with
 * H(k') = H_ii + H_{i,i+1} e^{ik'Lz} + H_{i,i-1} e^{-ik'Lz}; E_out is n_k x n,
 * ascending per k'.
 */
int pwqt_bands(pwqt_ctx* ctx, int n_k, const double* k, double* E_out);

/*
 * CUDA-event timing of the block-sweep kernels (the dominant cost, Sec. 3.2
 * system): with enable != 0 the block sweep of every batch (all its node and panel
 * launches) is bracketed by events on the stream it runs on and its duration is
 * accumulated.  Outputs (any may be NULL): total milliseconds, number of timed
 * sweeps, and their algorithmic flops, (56/3) N n^3 real flops per energy (complex LU 8/3 n^3 + solve for
 * X_i 8 n^3 + Schur product 8 n^3 per node).  reset != 0 zeroes the counters after
 * reading them.  Timing serialises the host with each sweep launch, and a mixed
 * batch that otherwise runs as two halves on two streams runs them one after the
 * other while timing is enabled, so that each launch's event time is its own.
 */
int pwqt_profile(pwqt_ctx* ctx, int enable, double* sweep_ms, long long* sweep_launches,
                 double* sweep_flops, int reset);

/*
 * Change the refinement stopping rule of the mixed path for later solves (the
 * pwqt_opts fields ir_tol and ir_max_iters; 0 selects the defaults 1e-10 and 40).
 * Errors: PWQT_ERR_INVALID_ARG for a negative or non-finite value.
 */
int pwqt_set_refinement(pwqt_ctx* ctx, double ir_tol, int ir_max_iters);

/*
 * Refinement phases of the mixed path recorded while pwqt_profile is enabled
 * (same reset): total milliseconds of the residual evaluations (B - A c, Sec. 3.2
 * system, of the kind set by pwqt_set_residual) and of the correction solves with the stored
 * complex64 factors, and the number of batched refinement iterations.  Any
 * pointer may be NULL.
 */
int pwqt_profile_refinement(pwqt_ctx* ctx, double* residual_ms, double* correction_ms, long long* iterations);

/*
 * Refinement residual of the mixed path (Sec. 3.2 system, r = B - A c; the paper
 * solves in FP64 directly and has no counterpart):
 *   PWQT_RESIDUAL_SLICED (default): FP64-accurate products on the bf16 tensor
 *     cores -- operands cut into 7-bit integer slices whose products the tensor
 *     cores sum exactly; residual error ~3e-12 ||B|| on the block-512 workload.
 *     Its slice panels take (N + 1) x 44 MB per system at n = 512 (built on the
 *     first mixed solve of a system, kept with it).
 *   PWQT_RESIDUAL_FLOAT_FLOAT: float-float arithmetic on the FP32 pipes
 *     (~48-bit significand; floor ~4e-10 ||B|| at block 512).
 * Errors: PWQT_ERR_INVALID_ARG for any other value.
 */
/*
 * Slice-product residual launches recorded while pwqt_profile is enabled (same
 * reset; the paper has no counterpart): CUDA-event milliseconds of the launches
 * (summed over the halves of a mixed batch), the method's complex multiply-adds
 * (3 N n^2 per solution column and evaluation), the bf16 MMA flops of the 34 kept
 * slice products, and the launch count.  Any pointer may be NULL.
 */
int pwqt_profile_residual(pwqt_ctx* ctx, double* ms, double* cmacs, double* mma_flops, long long* launches);
/*
 * Correction solves of the mixed path recorded while pwqt_profile is enabled (same
 * reset; the paper has no counterpart): CUDA-event milliseconds of the correction
 * launches (summed over the halves of a mixed batch, the same figure as the correction
 * time of pwqt_profile_refinement), the method's complex multiply-adds (3 N n^2 per
 * refining column: the products with L_i and X_i and the two triangular solves), and
 * the launch count.  Any pointer may be NULL.
 */
int pwqt_profile_correction(pwqt_ctx* ctx, double* ms, double* cmacs, long long* launches);

#define PWQT_RESIDUAL_SLICED       0
#define PWQT_RESIDUAL_FLOAT_FLOAT  1
int pwqt_set_residual(pwqt_ctx* ctx, int kind);

/*
 * pwqt_solve_noalloc -- the FP64 solve without any device allocation.
 * The paper has no counterpart; this entry point exists for callers that cannot
 * call cudaMalloc while they solve: code embedded in a host program that owns the
 * device-memory budget (its own pool allocator or a hard quota), or a service
 * whose request path must not allocate because cudaMalloc synchronises the device
 * and can fail under fragmentation.  Everything the call needs beyond the
 * caller's inputs and outputs lives in one static device array of 32 MiB that
 * every GPU loading the library holds until the process exits.
 *   - Inputs: the context's assembled system `sys` (pwqt_set_extrinsic) and its
 *     cached self-energies: call pwqt_prepare_leads (which allocates) for these
 *     energies first, else PWQT_ERR_STATE.  E is host memory, n_E <= 64.
 *   - Outputs: caller-owned DEVICE buffers T, R, T_ds [n_E], node_n [n_E*N*2]
 *     (required) and status [n_E] (may be NULL); same meaning as pwqt_solve.
 *   - Requests whose work panels (N n (n+m) complex128 per energy plus n x n
 *     blocks) exceed the 32 MiB return PWQT_ERR_INVALID_ARG and compute nothing.
 *   - The first call on a device, even one with n_E = 0, looks up the array's
 *     device address on that device (with the device current).  Under CUDA's
 *     lazy module loading that lookup also loads the library's module there and
 *     commits the 32 MiB, so this first call is the one that can allocate (and
 *     fail under a quota): make it once at start-up, before any stream capture,
 *     e.g. with n_E = 0.  Every call makes the context's device current for its
 *     duration and restores the caller's current device before it returns.  The
 *     call enqueues on `stream` (a cudaStream_t, NULL = legacy default stream)
 *     and returns after the stream has finished the work.
 *   - All calls share the array and it keeps the previous call's contents; the
 *     call re-initialises what must start defined.  Calls that overlap on the GPU
 *     (other host threads or streams at the same time) race on it: serialise them.
 */
int pwqt_solve_noalloc(pwqt_ctx* ctx, int sys, int n_E, const double* E, double* T, double* R,
                       double* T_ds, double* node_n, int* status, void* stream);

/*
 * Utility / test entry point: C[b] -= A[b] B[b] for b < batch on the tensor cores
 * (the library's complex64 3xTF32 GEMM of the mixed-precision sweep; the paper
 * has no counterpart).  Host arrays, row-major complex64 interleaved (float[2]),
 * batch entries stored back to back (M*lda, K*ldb, M*ldc complex each);
 * leading dimensions in complex elements.  Allocates and frees its own device
 * copies.  Errors: PWQT_ERR_INVALID_ARG, PWQT_ERR_OOM, PWQT_ERR_CUDA.
 */
int pwqt_cgemm_c64(int batch, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                   float* C, int ldc);

/*
 * Density-matrix route to the electron density (Sec. 3.3, Eq. density_matrices
 * and Eq. density_3d_fast).  Each system keeps, on the device, the density-matrix
 * blocks that the density needs: rho_d[a] (node a with itself, N blocks) and
 * rho_u[a] (node a with node a+1, N-1 blocks), n x n complex128 each,
 *     rho_d[a]_{alpha beta} = sum_{E, gamma} w_E g_gamma f_gamma conj(c_{a alpha}) c_{a beta}
 *     rho_u[a]_{alpha beta} = sum_{E, gamma} w_E g_gamma f_gamma conj(c_{a alpha}) c_{a+1 beta}
 * over the injected modes gamma of every accumulated energy, g = 2/|dE/dk| and
 * f = f_FD(E - mu_s) for source-injected modes, f_FD(E - mu_d) for drain-injected
 * ones, f_FD(x) = 1/(1 + e^{x/kT}) (a step for kT = 0).  pwqt_set_extrinsic
 * discards a system's density.
 *
 * pwqt_density_reset: zero (allocating on first use, 2 N n^2 complex128) the
 * density of system `sys`.  Errors: PWQT_ERR_STATE (unknown system), PWQT_ERR_OOM.
 */
int pwqt_density_reset(pwqt_ctx* ctx, int sys);

/*
 * Solve system `sys` at the n_E energies E (host) exactly as pwqt_solve with
 * `precision`, and add each solution's rank-m contribution to the system's
 * density (FP64 kernels); w (host, n_E) are the energy quadrature weights.  The
 * first call after pwqt_set_extrinsic starts from zero.  status (host, n_E, may
 * be NULL) receives the PWQT_ST_* bits of each energy; energies whose contacts
 * fail the mode count contribute nothing.  Errors: as pwqt_solve, and
 * PWQT_ERR_INVALID_ARG for NULL E / w, a non-finite weight or mu, or kT < 0.
 */
int pwqt_accumulate_density(pwqt_ctx* ctx, int sys, int n_E, const double* E, const double* w,
                            double mu_s, double mu_d, double kT, int precision, int* status);

/*
 * Copy the density matrix of system `sys` to the host: rho_d (N x n x n complex)
 * and rho_u ((N-1) x n x n complex), row-major interleaved; either may be NULL.
 * Errors: PWQT_ERR_STATE if nothing has been accumulated since pwqt_set_extrinsic.
 */
int pwqt_get_density_matrix(pwqt_ctx* ctx, int sys, double* rho_d, double* rho_u);

/*
 * Electron density n(r) on a real-space grid from the accumulated density
 * matrix (Eq. density_3d_fast).  On the element between nodes e and e+1
 * (e < N-1) the grid points are x_j = j Lx / nx (j < nx; only x = 0 for a
 * dim == 1 cell) and z = z_e + (q + 1/2) Lz / nz (q < nz).  n_r (host) receives
 * (N-1) x nx_eff x nz doubles, index (e * nx_eff + j) * nz + q, nx_eff = nx
 * (dim 2) or 1 (dim 1).  1 <= nx, nz <= 4096.  Errors: PWQT_ERR_STATE (no
 * density yet), PWQT_ERR_INVALID_ARG, PWQT_ERR_OOM.
 */
int pwqt_density_grid(pwqt_ctx* ctx, int sys, int nx, int nz, double* n_r);

/*
 * Transmission from the Green's function (Sec. 3.2: G = [E M - H - Sigma]^{-1}, the
 * NEGF alternative to the wave-function solve): T(E) = Tr[Gamma_d G_{N1} Gamma_s
 * G_{N1}^H], Gamma_c = i (Sigma_c - Sigma_c^H), with G_{N1} from the FP64 block sweep
 * with the identity injected at the first node.  Needs no mode decomposition at the
 * drain: it cross-checks the T of pwqt_solve (the two agree to rounding).  Host
 * arrays: E, T [n_E]; status [n_E] (may be NULL) receives the PWQT_ST_* bits.
 * Work per energy ~ the FP64 sweep with n injected columns.  Errors: as pwqt_solve.
 */
int pwqt_transmission_caroli(pwqt_ctx* ctx, int sys, int n_E, const double* E, double* T, int* status);

/*
 * Diagonal blocks of the retarded Green's function G = [E M - H - V^e - Sigma]^{-1}
 * (Sec. 3.2, the NEGF form of the open-boundary problem; Sigma = Sigma_s + Sigma_d on
 * the end nodes) by the recursive Green's-function recursion over the nodes: the
 * FP64 block sweep's forward elimination with [U_i | I] at every node gives X_i and
 * the left-connected g_i = S_i^{-1}; the backward pass forms G_{N-1} = g_{N-1},
 * G_i = g_i + (X_i G_{i+1})(U_i^H g_i).  Outputs (host, caller-owned):
 *   node_dos [n_E x N]: -(2/pi) Im Tr G_ii, the node spectral density; in a
 *       ballistic device it equals the sum of the source- and drain-injected node
 *       densities node_n of pwqt_solve (Sec. 3.3), with no mode decomposition inside
 *       the device;
 *   G_diag [n_E x N x n x n x 2] (may be NULL): the blocks G_ii, row-major,
 *       complex128 interleaved;
 *   status [n_E] (may be NULL): the PWQT_ST_* bits of the contacts and the sweep.
 * Work per energy ~51 N n^3 real flops (2.7x the mode-resolved FP64 sweep), device
 * memory ~N n^2 32 bytes per energy of a batch.  Errors: as pwqt_solve.
 */
int pwqt_green_diagonal(pwqt_ctx* ctx, int sys, int n_E, const double* E, double* node_dos, double* G_diag, int* status);

/*
 * Energy integrals by adaptive Simpson quadrature (Sec. 3.3: the density integral
 * is evaluated adaptively to a tolerance, with the error estimated on the node
 * density; Eq. current: the ballistic current with the same method).  Integrands:
 *   PWQT_INTEGRAND_CURRENT: (2e^2/h) (T_sd(E) f(E - mu_s) - T_ds(E) f(E - mu_d)), so
 *       that result[0] is the source-to-drain current in A for energies in eV (the
 *       Landauer form of Eq. current);
 *   PWQT_INTEGRAND_NODE_DENSITY: n^s[i](E) f(E - mu_s) + n^d[i](E) f(E - mu_d) per
 *       node (the node densities of pwqt_solve), result[N].
 * f(x) = 1/(1 + e^{x/kT}) (a step for kT = 0).  [E_lo, E_hi] starts as min_pieces
 * equal intervals; an interval of length h is accepted when its one- and two-panel
 * Simpson estimates S1, S2 differ by at most 15 tol h / (E_hi - E_lo) (max norm over
 * the components) and contributes S2 + (S2 - S1)/15; otherwise both halves are
 * examined.  Each refinement round solves all the energies it needs in one batched
 * pwqt_solve with `precision`.  After max_evals solved energies (or at intervals
 * 2^-40 of the range) open intervals are accepted as they stand.
 *   err_est  : sum over intervals of max|S2 - S1| / 15 (may be NULL)
 *   n_evals  : energies solved (may be NULL)
 *   energies, weights (may be NULL): the quadrature points, ascending, and their
 *       weights (the integral of any other per-energy quantity is sum w g(E), e.g.
 *       pwqt_accumulate_density with these weights); at most max_points are written,
 *       n_points receives the full count.
 * Errors: PWQT_ERR_STATE (unknown system), PWQT_ERR_INVALID_ARG, and those of
 * pwqt_solve.
 */
#define PWQT_INTEGRAND_CURRENT                0
#define PWQT_INTEGRAND_NODE_DENSITY           1
#define PWQT_INTEGRAND_NODE_DENSITY_JACOBIAN  2   /* result[2N]: the node density, then the same
                                                     with -df/dE in place of f (Eq. density_jacobian) */
int pwqt_integrate(pwqt_ctx* ctx, int sys, int integrand, double E_lo, double E_hi, double mu_s, double mu_d,
                   double kT, double tol, int min_pieces, int max_evals, int precision, double* result,
                   double* err_est, int* n_evals, double* energies, double* weights, int* n_points,
                   int max_points);

/*
 * Self-consistent potential (Sec. 4) on a 1D finite-element model of the non-linear
 * Poisson equation (Eq. nonlin_poisson_fem) along z, on the node hats f_i:
 *     (kappa S + gamma M) U = gamma M U_gate + alpha M (n[U] - n_dop),
 * S_ij = int f_i' f_j', M_ij = int f_i f_j (tridiagonal, node spacing Lz), U the
 * electron potential energy (eV) on the N nodes of system `sys`, held at U[0] and
 * U[N-1] (the contacts), n the node density per nm integrated over [E_lo, E_hi]
 * with f_FD (pwqt_integrate, tolerance tol_int).  Newton-Raphson (Eq. newton_poisson)
 * with the semi-classical Jacobian kappa S + gamma M + alpha M diag(d), d the node
 * density integrated with -df/dE (Eq. density_jacobian); the Newton outputs and
 * steps of the last diis_window iterates form the DIIS subspace (least squares by
 * SVD, singular values below 1e-10 of the largest dropped) whose extrapolation is the
 * next potential (diis_window <= 1: plain Newton).  Stops when the l2 norm of the
 * Newton step is <= tol_sc (eV).
 *   U       in: the starting potential (N values, ends fixed); out: the result.
 *   history (may be NULL, max_iters values): the step norm of every iteration.
 *   iters   receives the iteration count; n_out (may be NULL): n at the result.
 * The system's extrinsic blocks are rebuilt every iteration (pwqt_set_extrinsic);
 * the contact self-energy cache is reused (the contacts do not move).  Returns
 * PWQT_ERR_STATE if not converged within max_iters (U holds the last iterate).
 */
typedef struct {
    double        kappa;       /* eV nm                                               */
    double        gamma;       /* eV / nm                                             */
    double        alpha;       /* eV nm per unit of the node density per nm           */
    const double* U_gate;      /* N values (eV)                                       */
    const double* n_dop;       /* N values, in the units of the node density per nm   */
} pwqt_poisson1d;

int pwqt_self_consistent(pwqt_ctx* ctx, int sys, const pwqt_poisson1d* model, double mu_s, double mu_d,
                         double kT, double E_lo, double E_hi, double tol_int, double tol_sc, int max_iters,
                         int diis_window, int precision, double* U, double* history, int* iters,
                         double* n_out);

/*
 * Serving loop (continuous admission of solve requests).  A server owns one
 * context per catalog basis, each with its own CUDA stream and host worker thread:
 * requests on different bases run on the device at the same time, requests on one
 * basis in arrival order.  A request starts when the estimated working sets of the
 * running requests plus its own fit the device-memory budget; intrinsic blocks,
 * the contact self-energy cache, factor workspaces and the last 8 potentials per
 * basis stay resident between requests.  The paper has no serving layer; each
 * request is the solve of Sec. 3.2-3.4 exactly as pwqt_solve_dev computes it.
 */
typedef struct pwqt_server pwqt_server;

typedef struct {
    int    device;             /* CUDA device ordinal                                  */
    size_t hbm_budget_bytes;   /* admission budget; 0: 70 % of the free device memory  */
    int    queue_capacity;     /* queued requests before submit returns BUSY; 0: 4096  */
    double ir_tol;             /* as pwqt_opts                                         */
    int    batch;              /* as pwqt_opts                                         */
} pwqt_server_opts;

typedef struct {
    int           basis;       /* catalog id given to pwqt_server_add_basis           */
    int           n_nodes;     /* N >= 2                                               */
    const double* U;           /* N node potentials (eV), copied at submission         */
    int           n_E;         /* >= 1                                                 */
    const double* E;           /* energies (eV), copied at submission                  */
    int           precision;   /* PWQT_FP64 | PWQT_MIXED | PWQT_FP32                   */
    /* host outputs, caller-owned, written before pwqt_server_wait returns OK; each may
       be NULL; sizes and meaning as pwqt_solve (node_n: n_E * N * 2)                  */
    double *T, *R, *T_ds;
    int*    n_open;
    double* node_n;
    double* resid;
    int *   iters, *status;
} pwqt_request;

/* Errors: PWQT_ERR_NO_DEVICE, PWQT_ERR_INVALID_ARG (device ordinal), PWQT_ERR_CUDA. */
int pwqt_server_create(pwqt_server** out, const pwqt_server_opts* opts);

/* Add a catalog basis: a context assembled as pwqt_assemble_intrinsic; n_out
   receives its block size.  Errors: as pwqt_assemble_intrinsic; INVALID_ARG for a
   basis id already present. */
int pwqt_server_add_basis(pwqt_server* srv, int basis, const pwqt_cell* cell, const pwqt_formfactor* ff,
                          double gcut, int n_bands, int* n_out);

/* Queue a request; ticket receives its id.  The output buffers must stay valid
   until pwqt_server_wait has returned PWQT_OK for the ticket.  Errors: INVALID_ARG
   (unknown basis, sizes, non-finite input), PWQT_ERR_BUSY (queue full),
   PWQT_ERR_OOM (working set larger than the whole budget). */
int pwqt_server_submit(pwqt_server* srv, const pwqt_request* req, long long* ticket);

/* Wait up to timeout_s seconds (< 0: without limit) for a request.  PWQT_OK: done,
   result receives the solve's return code (PWQT_OK or a PWQT_ERR_*, message in
   pwqt_server_last_error), latency_s the seconds from submission to completion,
   and the ticket is released.  PWQT_ERR_TIMEOUT: still queued or running (ask
   again).  PWQT_ERR_INVALID_ARG: unknown or already collected ticket. */
int pwqt_server_wait(pwqt_server* srv, long long ticket, double timeout_s, int* result, double* latency_s);

/* Completed requests since the last reset, latency percentiles over them (nearest
   rank), and the largest admitted working-set sum; reset != 0 restarts them. */
int pwqt_server_stats(pwqt_server* srv, long long* completed, double* p50_s, double* p99_s,
                      size_t* peak_admitted_bytes, int reset);

/* Continuous batching since the last reset of pwqt_server_stats: batched solves
   run, requests they held, and the largest batch.  Requests queued on one basis
   with the same node count and precision share a batched solve (up to 8 distinct
   potentials, within the budget); the paper has no counterpart. */
int pwqt_server_batch_stats(pwqt_server* srv, long long* batches, long long* requests, long long* largest);

/* Message of the last failure on this server (valid until the next failure). */
const char* pwqt_server_last_error(pwqt_server* srv);

/* Finish the queued requests, stop the workers, release every context.  NULL is
   accepted. */
int pwqt_server_destroy(pwqt_server* srv);

/* Launch counters of the library's own kernels since the last reset. */
int pwqt_kernel_launches(pwqt_ctx* ctx, long long* count, int reset);

#ifdef __cplusplus
}
#endif
#endif /* PWQT_H */
