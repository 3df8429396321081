/*
 * wd.h -- C ABI of a GB300 (sm_103a) mixed-precision Wilson-Dirac solver.
 *
 * The library solves D_W xi = eta (Eq. 3) for the Wilson matrix of Eq. 1,
 *   D_W = 1 - kappa * H,
 *   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                       + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ],
 * through the even-odd system of Eqs. 4-5 (A = 1 - kappa^2 H_eo H_oe on even
 * sites), with the FP64 iterative refinement of Algorithms 2-3 around the
 * rescaled low-precision BiCGStab of Algorithms 4-5.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - dims = {Lx, Ly, Lz, Lt}; every extent even and >= 2.
 * - Lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t)); parity of a site
 *   is (x+y+z+t) mod 2, 0 = even.
 * - Dirac matrices: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1..3),
 *   gamma_4 = diag(1, 1, -1, -1); this is the representation whose
 *   (1 - gamma_1) is printed in Eq. 2.
 * - Boundary phases bc[mu] in {+1, -1} multiply hops that wrap around the
 *   lattice in direction mu; default {1, 1, 1, -1} (antiperiodic in time).
 * - Host / "lexicographic" layouts, all float64 with (re, im) innermost:
 *     gauge  U[mu][s][a][b][2] = (U_mu(x_s))_ab,  mu = 0..3 is x, y, z, t;
 *     vector psi[s][spin][colour][2] (24 doubles per site).
 * - Packed layouts (device only, produced by wd_pack / consumed by
 *   wd_unpack): one parity of a vector is V/2 sites of 24 reals in the
 *   precision's storage type, stored as 16-byte units with the site index
 *   fastest: unit u of site h sits at byte 16 * (u * V/2 + h). Site h of
 *   parity p is the lexicographic site 2h or 2h+1 whose parity is p.
 *   wd_vector_bytes() gives the size of one parity vector; a "full" packed
 *   vector is the even parity followed by the odd parity.
 * - All device work is enqueued on the caller's CUDA stream (a
 *   cudaStream_t passed as void*, NULL = legacy default stream). Entry
 *   points that return a result synchronize that stream only when stated.
 * - Return value: a wd_status code. No C++ exception crosses this ABI. The
 *   text of the last failure of a handle is in wd_last_error().
 * - Ownership: the library copies every input; callers keep their buffers.
 *   The handle owns its device workspaces (allocated on first use, freed
 *   by wd_destroy).
 * - Thread safety: one handle must not be used from two host threads at once.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_handle wd_handle;

/* Status codes. */
enum wd_status {
    WD_OK = 0,
    WD_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or state                      */
    WD_ERR_CUDA = 2,          /* a CUDA runtime call failed                            */
    WD_ERR_NOT_SU3 = 3,       /* 12-real links requested but U is not in SU(3)         */
    WD_ERR_NOT_CONVERGED = 4, /* iteration caps reached; best iterate returned         */
    WD_ERR_BREAKDOWN = 5,     /* (r*, v) = 0 or (t, t) = 0 in BiCGStab                 */
    WD_ERR_NONFINITE = 6,     /* a scalar of the recurrence became Inf or NaN          */
    WD_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                    */
    WD_ERR_NO_GAUGE = 8       /* wd_set_gauge has not been called                      */
};

/* Storage precisions of packed vectors and links. Arithmetic is FP32 for
 * FP32/FP16/BF16 storage and FP64 for FP64 storage. */
enum wd_prec { WD_FP64 = 0, WD_FP32 = 1, WD_FP16 = 2, WD_BF16 = 3 };

/* Link formats: 18 reals (full 3x3) or 12 reals (two rows; the third row is
 * rebuilt as the complex conjugate of the cross product of the first two,
 * exact for SU(3)). */
enum wd_recon { WD_RECON_12 = 12, WD_RECON_18 = 18 };

/* Operators of wd_apply (Eq. 1 and Eq. 4). */
enum wd_op {
    WD_OP_HOP_EO = 0, /* out(even) = H_eo in(odd)                                   */
    WD_OP_HOP_OE = 1, /* out(odd)  = H_oe in(even)                                  */
    WD_OP_EO_A = 2,   /* out(even) = in - kappa^2 H_eo H_oe in   (bracket of Eq. 4) */
    WD_OP_FULL = 3    /* out(full) = D_W in (full packed vectors, Eq. 1)            */
};

/* Where a caller's buffer lives. */
enum wd_where { WD_HOST = 0, WD_DEVICE = 1 };

/* Solver schemes (Sec. 3 and Table 2). */
enum wd_scheme {
    WD_FP64_BICGSTAB = 0,     /* BiCGStab (Alg. 4 with gamma = 1) entirely in FP64       */
    WD_MIXED_FP32 = 1,        /* Alg. 2 refinement, FP32 inner BiCGStab without rescaling */
    WD_MIXED_FP16_PLAIN = 2,  /* Alg. 2 refinement, FP16 inner without rescaling          */
    WD_MIXED_FP16 = 3,        /* Alg. 3 refinement, FP16 inner Alg. 4 / Alg. 5            */
    WD_MIXED_BF16 = 4,        /* as WD_MIXED_FP16 with BF16 storage (Sec. 7 outlook)      */
    WD_MIXED_FP16_LEARNED = 5 /* as WD_MIXED_FP16, inner BiCGStab on A M with the learned
                                 right preconditioner M (wd_precond_set first)            */
};

/* Knobs of Algorithms 2-5. wd_solve_params_default() fills the values a
 * scheme uses by default. */
typedef struct wd_solve_params {
    double s;             /* Alg. 3: norm of the rescaled outer residual y (Alg. 2: 1)      */
    double sigma;         /* Alg. 4: norm of the inner residual after rescaling; 0 = none  */
    double sigma_lambda;  /* Alg. 5: norm of the rescaled inner solution                    */
    double inner_eps;     /* inner stop: |r|/gamma' <= inner_eps * |y~| (eps, not eps^2)    */
    double omega0;        /* omega_0 of the BiCGStab prescription (0.7)                     */
    int recalc_gamma;     /* gamma := |r_stored| / g  instead of sigma / g                   */
    int rescale_x;        /* Alg. 5 (solution rescaling)                                     */
    int use_shat;         /* Alg. 3: correct with s^ = |single(y~)| instead of s             */
    int x_is_guess;       /* x holds an initial guess (restart from a previous solution)    */
    int max_outer;        /* cap on refinement trips                                         */
    int max_inner;        /* cap on low-precision matrix-vector products per inner solve    */
    int recon;            /* link format of the inner operator: 12 or 18                     */
    int ftz;              /* flush subnormal low-precision values to zero on store           */
    int iters_per_sync;   /* inner iterations captured per CUDA-graph launch                 */
    double* history;      /* optional host array of history_cap entries of 4 doubles, filled
                             for a solve of one system with one right-hand side (wd_solve)
                             with the convergence history:
                             {kind, matvecs, residual, nonzeros}; kind 1 = a refinement trip
                             (residual = |b^ - A x| / |eta| in FP64 at its start, nonzeros =
                             nonzero reals of its low-precision input), kind 0 = an inner
                             BiCGStab iteration (residual = its |r| / gamma' mapped to the
                             outer scale, (|r| / gamma') |r_outer| / (s^ |eta|)); matvecs =
                             low-precision matvecs so far. NULL = none                       */
    int history_cap;      /* entries `history` holds                                         */
    int fused_rescale;    /* 1 (default): Alg. 4's rescaling r := (sigma / g) r is applied as r
                             is formed, with g~^2 = (s,s) - 2 Re(conj(omega) (t,s))
                             + |omega|^2 (t,t) predicted from the dot products that give
                             omega (equal to |s - omega t|^2 in exact arithmetic); g itself,
                             gamma and the stopping test still use the norms of the formed r.
                             Saves one pass over r and its norms per iteration. 0: a separate
                             pass after g is known. Alg. 5 always uses the separate pass.   */
} wd_solve_params;

/* Counters of one solve. */
typedef struct wd_solve_stats {
    int status;                /* wd_status of the solve                                 */
    int outer_iterations;      /* refinement trips (Alg. 2/3 loop bodies)                */
    int inner_iterations;      /* BiCGStab iterations summed over trips                  */
    int inner_matvecs;         /* low-precision applications of A (2 per iteration)     */
    int outer_matvecs;         /* FP64 applications of A (true residuals)                */
    double true_residual;      /* |eta - D_W xi| / |eta|, computed in FP64 on the GPU    */
    double outer_residual;     /* last |b^ - A xi_e| / |eta| of the refinement           */
    double elapsed_ms;         /* device time of the whole solve (CUDA events)           */
    long long first_inner_nonzeros; /* nonzero reals of the first low-precision input    */
    long long kernel_launches; /* device kernels this call launched (graph nodes included) */
    int history_len;           /* entries written to params->history                     */
} wd_solve_stats;

/* Create a lattice handle. dims: 4 even extents >= 2, Lx*Ly*Lz*Lt/2 < 2^31.
 * kappa: hopping parameter of Eq. 1. bc: 4 boundary phases in {+1,-1}, or
 * NULL for {1,1,1,-1}. On success *out owns no device memory yet. */
int wd_create(const int dims[4], double kappa, const int bc[4], wd_handle** out);

/* Release the handle and all its device memory (synchronizes the device). */
int wd_destroy(wd_handle* h);

/* Load the gauge field U (Sec. 2, links U_mu(x) on x -> x+mu). U is in the
 * host layout above, 4*V*18 doubles, host or device memory as `where` says.
 * The library keeps an FP64 copy on the device and builds each packed link
 * format on first use. Synchronizes the default stream. */
int wd_set_gauge(wd_handle* h, const double* U, int where);

/* Largest |U U^+ - 1| entry and |det U - 1| over all links of the loaded
 * gauge field (FP64). 12-real formats are refused when either exceeds 1e-6. */
int wd_gauge_unitarity(wd_handle* h, double* max_unitarity_dev, double* max_det_dev);

/* Add the clover (Sheikholeslami-Wohlert) term to the matrix of the handle:
 * D_sw = C - kappa H with the site-local 12 x 12 Hermitian blocks
 *   C(x) = 1 - c_sw kappa sum_{mu<nu} sigma_mu_nu (x) Fh_mu_nu(x),
 * sigma_mu_nu = (i/2) [gamma_mu, gamma_nu] (the gamma matrices of this
 * header), Fh_mu_nu = traceless part of (Q_mu_nu - Q_mu_nu^+) / (8 i) and
 * Q_mu_nu(x) the four plaquettes of the mu-nu plane with a corner at x, each
 * traversed mu-then-nu; the links are periodic. The paper uses the plain
 * Wilson matrix and names the clover matrix as the next one to study
 * (Sec. 7); its even-odd system (Eqs. 4-5) takes the blocks as D_ee, D_oo:
 *   A = 1 - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe,
 *   b^ = C_ee^-1 (eta_e + kappa H_eo C_oo^-1 eta_o),
 *   xi_o = C_oo^-1 (eta_o + kappa H_oe xi_e).
 * Afterwards wd_apply (WD_OP_EO_A, WD_OP_FULL) and the solvers use D_sw (the
 * hopping operators WD_OP_HOP_* are unchanged); the refinement stops when
 * |b^ - A xi_e| <= tol |eta| / (1 + 12 |c_sw| kappa), which bounds the full
 * residual |eta - D_sw xi| = |C_ee (b^ - A xi_e)| by tol |eta|. C and C^-1
 * are computed in FP64 on the device (Gauss-Jordan per site) and converted
 * to other precisions on first use; wd_set_gauge rebuilds them. c_sw = 0
 * removes the term. Not available with WD_MIXED_FP16_LEARNED. Requires
 * wd_set_gauge first (WD_ERR_NO_GAUGE); WD_ERR_INVALID_ARG for a non-finite
 * c_sw or a singular block. */
int wd_set_clover(wd_handle* h, double csw);

/* Arithmetic of the hopping term H on FP16 storage (Sec. 5): bits = 32 (the
 * default) widens the stored FP16 values and computes the projection's
 * products, the SU(3) multiplies and the sum over the eight directions in
 * FP32; bits = 16 computes all of them in FP16 (packed half2 operations, one
 * rounding per operation), the arithmetic of the paper's _Float16 build; the
 * FP16 sum is held scaled by an exact power of two at or below |a| / 8 (a the
 * coefficient of H in the operation) so that it keeps the output's range. The
 * epilogue of a fused kernel (out = a H in + b y + c z, clover blocks, dot
 * products) stays FP32 and every reduction FP64 in both. Applies to
 * everything the handle does afterwards with WD_FP16 storage: wd_apply,
 * wd_apply_eo_noalloc and the inner solves of WD_MIXED_FP16,
 * WD_MIXED_FP16_PLAIN and WD_MIXED_FP16_LEARNED. WD_ERR_INVALID_ARG for any
 * other bits. wd_get_arith returns the current setting (0 for a null handle). */
int wd_set_arith(wd_handle* h, int bits);
int wd_get_arith(const wd_handle* h);

/* Limit of the bounded device-side waits (mbarrier waits on tensor-core
 * results and on bulk copies into shared memory) of the handle's kernels, in
 * wait rounds; rounds < 0 restores the default (4,194,304 rounds, about a
 * second). Not a feature of the paper: it exists to exercise the timeout
 * path, which a healthy GPU never takes. A wait that runs out raises a
 * device flag; the kernel then waits, with the default bound, for its own
 * copies and tensor-core operations in flight, frees its tensor memory and
 * returns, and the call returns WD_ERR_TIMEOUT (wd_precond_apply, wd_solve,
 * wd_solve_batch: the status of every right-hand side). rounds = 0 makes
 * every such wait give up at once. The handle stays usable. */
int wd_set_wait_limit(wd_handle* h, long long rounds);

/* Bytes of one packed parity vector in precision `prec` (24 * V/2 reals). */
size_t wd_vector_bytes(const wd_handle* h, int prec);

/* Pack the sites of parity `parity` of the device FP64 lexicographic vector
 * `lex` (24*V doubles) into the device buffer `packed` (wd_vector_bytes). */
int wd_pack(wd_handle* h, int prec, int parity, const double* lex, void* packed, void* stream);

/* Scatter the packed parity vector back into the device FP64 lexicographic
 * vector `lex`; sites of the other parity are left untouched. */
int wd_unpack(wd_handle* h, int prec, int parity, const void* packed, double* lex, void* stream);

/* Apply an operator (enum wd_op) in storage precision `prec` with link
 * format `recon` to the packed device vector `in`, writing packed `out`
 * (in and out must not overlap). Arithmetic as in enum wd_prec. */
int wd_apply(wd_handle* h, int prec, int recon, int op, const void* in, void* out, void* stream);

/* wd_apply on nrhs right-hand sides at once: `in` and `out` hold nrhs packed
 * vectors of the operator's kind (parity vectors, or full vectors for
 * WD_OP_FULL) back to back, right-hand side r at r times the vector size. The
 * kernels serve all right-hand sides in one launch per hop (the batched form
 * of the 12 spin-colour sources); with FP16 arithmetic each thread may apply
 * its site's links to K right-hand sides (wd_tune, wd_set_rhs_per_thread).
 * 1 <= nrhs <= 1024. */
int wd_apply_batch(wd_handle* h, int prec, int recon, int op, int nrhs, const void* in, void* out, void* stream);

/* Right-hand sides per thread of the FP16-arithmetic hop (wd_set_arith(16),
 * FP16 storage) with link format `recon`, as wd_tune would choose them:
 * k_plain for the plain hop, k_reducing for the hop with fused epilogue and
 * dot products (1..12; a batch uses the largest divisor of its nrhs up to
 * k), links_smem = 1 to stage the site's links in shared memory instead of
 * registers. The results are the same bits for every k (each right-hand
 * side is computed by the same operations); only the speed differs. Not a
 * feature of the paper. */
int wd_set_rhs_per_thread(wd_handle* h, int recon, int k_plain, int k_reducing, int links_smem);

/* out = in - kappa^2 H_eo H_oe in, exactly as wd_apply(h, prec, recon,
 * WD_OP_EO_A, ...), for callers that must not allocate device memory (code
 * that runs under a caching allocator owning all device memory, or code that
 * must not risk the implicit device synchronization of cudaMalloc/cudaFree).
 * The paper has no counterpart; it is a service of this library.
 * - Allocates nothing: the odd-site intermediate lives in a fixed 16 MiB
 *   array in the library's device memory, held on every GPU that loads the
 *   library until the process exits. A precision whose odd-site vector
 *   (wd_vector_bytes) exceeds 16 MiB is refused with WD_ERR_INVALID_ARG
 *   (FP16: up to 349,525 sites per parity, e.g. 24^3 x 48).
 * - The links of (prec, recon) must already exist: call wd_apply or wd_solve
 *   with them once before (building them allocates); otherwise
 *   WD_ERR_INVALID_ARG.
 * - With a clover term (wd_set_clover) the result is the clover operator
 *   in - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe in, as from wd_apply. Its blocks
 *   C^-1 in precision `prec` must already exist: one wd_apply(WD_OP_EO_A) or
 *   wd_solve in that precision after wd_set_clover builds them; otherwise
 *   WD_ERR_INVALID_ARG.
 * - Uses the kernel configuration wd_tune chose and the FP16 arithmetic of
 *   wd_set_arith, as wd_apply does, so both give the same bits.
 * - The first call on a device looks up the array's device address; make
 *   that first call outside any stream capture.
 * - All calls on a device share the array: calls that may overlap on the GPU
 *   (different streams without ordering) race and give wrong results. */
int wd_apply_eo_noalloc(wd_handle* h, int prec, int recon, const void* in, void* out, void* stream);

/* ---- Domain decomposition ------------------------------------------------
 * The global lattice is split into a grid of sub-lattices, one per process
 * (the paper runs 64 MPI processes, Sec. 6, and sums every global reduction
 * in FP64 across them, Sec. 5, Fig. 3). Each process creates a handle with
 * its LOCAL extents (every one even, so a site's parity is the same in local
 * and global coordinates; the global extent in mu is grid[mu] times the
 * local one), loads its local links (wd_set_gauge, local lexicographic
 * order) and calls wd_dd_set_partition. The hopping term H_pq of Eq. 1 on
 * the sub-lattice is then
 *   H = (interior hops, wd_dd_hop_interior) + (face hops, wd_dd_hop_faces),
 * the face hops built from half spinors the neighbours packed (wd_dd_pack)
 * and the caller moved (MPI, NCCL, or copies). Per direction mu with
 * grid[mu] > 1 there are 8 face buffers send[d] / recv[d], d = 2 mu + side:
 *   side 0: the lower face x_mu = 0 of `in`, (1 - gamma_mu) in, two spin rows;
 *           send[2 mu] goes to the neighbour at coords[mu] - 1, whose
 *           recv[2 mu] it becomes;
 *   side 1: the upper face x_mu = L_mu - 1 of `in`, U_mu(x)^+ (1 + gamma_mu) in;
 *           send[2 mu + 1] goes to the neighbour at coords[mu] + 1, whose
 *           recv[2 mu + 1] it becomes;
 * (coordinates modulo grid[mu]; with grid[mu] = 2 both go to the same
 * neighbour and must stay apart). A face buffer holds wd_dd_face_bytes(mu)
 * bytes: 12 reals of the storage precision per face site, real e of face
 * site f at element e * F + f, F = V_local / 2 / L_mu, f = the
 * lexicographic index of the three other local coordinates (lowest
 * direction fastest) halved. Buffers of directions that are not split are
 * ignored (may be NULL). The boundary phase bc[mu] of a hop that wraps
 * around the global lattice is applied by the packing process. Arithmetic
 * as in enum wd_prec. Not available with a clover term or the learned
 * preconditioner; on a split handle wd_apply, wd_solve, wd_solve_batch and
 * wd_precond_* return WD_ERR_INVALID_ARG. */

/* Declare this handle the sub-lattice at `coords` of a process grid `grid`
 * (grid[mu] >= 1, 0 <= coords[mu] < grid[mu]); the handle's boundary phases
 * bc are those of the global lattice. All grid[mu] = 1 undoes the split.
 * Packed links built before are rebuilt on next use. */
int wd_dd_set_partition(wd_handle* h, const int grid[4], const int coords[4]);

/* Bytes of one face buffer of direction mu in precision prec (0 on bad input). */
size_t wd_dd_face_bytes(const wd_handle* h, int prec, int mu);

/* Pack the faces of the packed device vector `in` (parity 1 - parity) that
 * the neighbours' hops onto output parity `parity` need, into the device
 * buffers send[0..7]. */
int wd_dd_pack(wd_handle* h, int prec, int parity, const void* in, void* const send[8], void* stream);

/* out = a * H_int in + b * y on the local sites of parity `parity` (y may be
 * NULL when b = 0), H_int the hops of Eq. 1 that stay inside the sub-lattice
 * (all of them in directions that are not split). Runs the kernels of
 * wd_apply; it reads no face buffer, so it may overlap the exchange. */
int wd_dd_hop_interior(wd_handle* h, int prec, int recon, int parity, const void* in, const void* y, double a,
                       double b, void* out, void* stream);

/* out += a * (hops of Eq. 1 that enter the sub-lattice through its faces),
 * from the received face buffers recv[0..7], on the local sites of parity
 * `parity`. After it, out = a * H in + b * y of the whole lattice restricted
 * to this sub-lattice. */
int wd_dd_hop_faces(wd_handle* h, int prec, int parity, const void* const recv[8], double a, void* out, void* stream);

/* Local FP64 part of the dot product (a, b) = sum_i conj(a_i) b_i over the
 * sites of one packed parity vector (Sec. 5: sums widened to FP64, the
 * global sum across processes is the caller's FP64 allreduce). out[0], out[1]
 * = real and imaginary part, host memory. Deterministic (fixed block order).
 * Synchronizes `stream`. */
int wd_vec_dot(wd_handle* h, int prec, const void* a, const void* b, double out[2], void* stream);

/* y = a x + b y for packed parity vectors, a and b complex ((re, im) pairs,
 * host memory), arithmetic as in enum wd_prec. */
int wd_vec_axpby(wd_handle* h, int prec, const double a[2], const void* x, const double b[2], void* y,
                 void* stream);

/* Result of wd_tune. */
typedef struct {
    int variant;          /* plain hop: kernel variant chosen (see wd_tune)                */
    int block;            /* plain hop: threads per block chosen                           */
    double us;            /* plain hop: its average launch time, microseconds              */
    double default_us;    /* plain hop: the default configuration (variant 4, 128 threads) */
    int candidates;       /* configurations timed per form                                 */
    int variant_reducing; /* hop with fused epilogue and dot products: variant chosen      */
    int block_reducing;   /* ... threads per block chosen                                  */
    double us_reducing;   /* ... its average launch time, microseconds                     */
    /* FP16 storage with FP16 arithmetic (wd_set_arith(16)) and nrhs > 1: the FP16-arithmetic
       hop over K right-hand sides per thread (the site's links loaded once for K), K a divisor of
       nrhs up to 12, links in registers or shared memory; 1, 0, 0 otherwise                  */
    int rhs_per_thread;           /* plain hop: K chosen                                       */
    int rhs_links_smem;           /* plain hop: 1 = links staged in shared memory             */
    double us16;                  /* plain hop: its average launch time, microseconds         */
    int rhs_per_thread_reducing;  /* hop with fused epilogue and dot products: K chosen       */
    int rhs_links_smem_reducing;  /* ... links in shared memory                               */
    double us16_reducing;         /* ... its average launch time, microseconds                */
    int candidates16;             /* FP16-arithmetic configurations timed per form            */
    int sites_per_thread;         /* plain FP16-arithmetic hop with K = 1: sites per thread
                                     chosen among 1, 2, 4 (grid-stride launch)                */
} wd_tune_result;

/* Autotune the hopping kernel H_eo (Eq. 1) of storage precision `prec` with
 * link format `recon` for batches of `nrhs` right-hand sides on this lattice,
 * separately for its two forms in the solvers (the plain hop, and the hop with
 * fused epilogue and dot products that ends each even-odd operator): times
 * every candidate kernel variant and block size on scratch vectors (2 warm-up
 * and 8 timed launches each, CUDA events on `stream`) and keeps the fastest
 * for every later wd_apply / wd_solve / wd_solve_batch of the handle in that
 * (prec, recon); captured solver graphs are rebuilt. Candidates:
 * variant 4 (one site per thread, loads one direction ahead; 64 and 128
 * threads, and 256 except for FP16), 1 (no look-ahead), 2 (two sites per
 * thread, FP32x2; not FP64),
 * and for 16-bit storage 3 (tiles staged in shared memory), 6 (FP32x2 column
 * pairs; 64, 128 threads, and 256 for BF16) and, with 12-real links, 5 (per-thread cp.async
 * ring). These are the kernels of FP32 arithmetic. With wd_set_arith(16) and
 * FP16 storage the FP16-arithmetic kernel runs instead (128 threads, one site
 * per thread); for nrhs > 1 wd_tune then also times it with K right-hand
 * sides per thread (every divisor K of nrhs up to 12; the site's 8 links are
 * loaded once for its K right-hand sides, in registers or in shared memory)
 * and, for K = 1, the plain hop with 1, 2 or 4 sites per thread, and keeps
 * the fastest for each form (wd_set_rhs_per_thread sets K
 * directly); a batch of nrhs right-hand sides then uses the largest divisor
 * of nrhs up to that K. Not a feature of the paper. Synchronizes `stream`;
 * allocates three scratch vectors of nrhs parity vectors. `out` may be NULL. */
int wd_tune(wd_handle* h, int prec, int recon, int nrhs, void* stream, wd_tune_result* out);

/* Fill `p` with the defaults of `scheme` (Table 2 rows; s = 128, sigma = 64
 * for WD_MIXED_FP16). */
int wd_solve_params_default(int scheme, wd_solve_params* p);

/* Solve D_W x = b to |b - D_W x| <= tol |b| (Alg. 3 + Alg. 4/5 around the
 * even-odd system, Eqs. 4-5). b and x are full-lattice FP64 vectors in the
 * host layout, in host or device memory (detected per pointer; host buffers
 * are copied in and out inside the call). params may be NULL (defaults of
 * the scheme); stats may be NULL. Synchronizes `stream` once per refinement
 * trip to read the outer residual norm, and at the end.
 * Returns WD_OK, WD_ERR_NOT_CONVERGED (x holds the best iterate),
 * WD_ERR_BREAKDOWN, WD_ERR_NONFINITE, or an argument / CUDA error. */
int wd_solve(wd_handle* h, const double* b, double* x, double tol, int scheme,
             const wd_solve_params* params, wd_solve_stats* stats, void* stream);

/* Solve several right-hand sides on several lattices in one batched launch
 * chain. For lattice i (0 <= i < n), nrhs[i] sources b[i] and solutions x[i]
 * are stored back to back (nrhs[i] full-lattice vectors each, device memory).
 * Links are read once per site for all right-hand sides of a lattice.
 * per_rhs_stats (optional) receives sum(nrhs) entries in order. */
int wd_solve_batch(int n, wd_handle* const* h, const int* nrhs, const double* const* b,
                   double* const* x, double tol, int scheme, const wd_solve_params* params,
                   wd_solve_stats* per_rhs_stats, void* stream);

/* ---- Learned right preconditioner M --------------------------------------
 * A linear, gauge-equivariant parallel-transport network with channels
 * 1 -> 12 -> 1 (not in the paper; its inner solve is the paper's Alg. 4 on
 * A M). One layer maps C_in to C_out quark-field channels:
 *   out[c](x) = sum_{k=0..8} sum_{c'} W[k][c][c'] (T_k in[c'])(x),
 * hop k = 0 is the identity; k = 1 + d for d = 2 mu transports from x + mu with
 * U_mu(x), and for d = 2 mu + 1 from x - mu with U_mu(x - mu)^+, with the
 * boundary phases of the Wilson matrix; W[k][c][c'] is a complex 4x4 spin
 * matrix. M maps even-site vectors to even-site vectors.
 * Weight layout (WD_PRECOND_FLOATS floats): layer 1 W1[k][c][s][t][re,im]
 * (c = hidden channel), then layer 2 W2[k][c][s][t][re,im]. The kernels use
 * the BF16-rounded weights with FP32 arithmetic. */
#define WD_PRECOND_FLOATS 6912

/* Load FP32 master weights (host or device memory); resets the Adam state. */
int wd_precond_set(wd_handle* h, const float* w, int where);

/* Copy the FP32 master weights out (host or device memory). */
int wd_precond_get(wd_handle* h, float* w, int where);

/* out = M in for packed even-site vectors in precision WD_FP32 (FP32 hidden
 * channels, FP32 18-real links) or WD_FP16 (BF16 hidden channels, FP16 12-real
 * links, as inside the WD_MIXED_FP16_LEARNED solve). */
int wd_precond_apply(wd_handle* h, int prec, const void* in, void* out, void* stream);

/* Training loss L = sum_i |M v_i - y_i|^2 / |y_i|^2 + mu |A M v_i - v_i|^2 / |v_i|^2
 * over n samples (v_i, y_i = A^{-1} v_i): packed FP32 even-site vectors stored
 * back to back in device memory. Writes L to *loss and, if grad is not NULL,
 * dL/dRe W + i dL/dIm W (flat weight layout, device memory) to grad.
 * Synchronizes `stream`. */
int wd_precond_grad(wd_handle* h, int n, const float* v, const float* y, double mu, float* grad, double* loss,
                    void* stream);

/* One Adam step (beta1 0.9, beta2 0.999) with learning rate lr on the loss of
 * wd_precond_grad; *loss receives the loss before the step. */
int wd_precond_train_step(wd_handle* h, int n, const float* v, const float* y, double mu, double lr, double* loss,
                          void* stream);

/* The learned part under the names of its specified interface. wd_precond_load
 * loads n = WD_PRECOND_FLOATS weights given as BF16 values (uint16 bit
 * patterns, host memory, the flat layout above): each is widened exactly to
 * FP32 and the result loaded as by wd_precond_set (Adam state reset).
 * WD_ERR_INVALID_ARG for another n. wd_precond_train runs `steps` >= 1 calls
 * of wd_precond_train_step on the same n samples; *loss (may be NULL)
 * receives the loss before the last step. Errors as those calls. */
int wd_precond_load(wd_handle* h, const void* weights_bf16, size_t n);
int wd_precond_train(wd_handle* h, int steps, int n, const float* v, const float* y, double mu, double lr,
                     double* loss, void* stream);

/* Arithmetic throughput probe (not a feature of the paper): launches one
 * kernel on `stream` that runs `iters` steps of 8 independent fused
 * multiply-add chains per thread on the FP64 (bits = 64), FP32 (32) or
 * packed FP16 (16) pipe, over 8 blocks of 256 threads per SM, and stores in
 * *flops the floating-point operations of the launch (2 per multiply-add and
 * lane). The caller times the launch (CUDA events on `stream`) to get the
 * rate that bounds a kernel limited by that pipe. `sink`: a device buffer of
 * at least 4 * 8 * SMs bytes the kernel may write. */
int wd_fma_probe(int bits, long long iters, void* sink, void* stream, double* flops);

/* Kernel timeline (not a feature of the paper; the library built with
 * -DWD_TIMELINE, libwd_timeline.so): from this call on, every block of the
 * solvers' hopping and vector kernels appends one record of four 64-bit words
 * to `blocks` and the last block of every grid reduction one record of ten
 * words to `phases` (device buffers owned by the caller; word 0 of each is
 * the record count, set it to 0; at most 2^24 block and 2^20 reduction
 * records are kept). Block record: (source line | kernel tag << 12 |
 * file-name hash << 16) << 32 | grid size << 8 | SM (the tag tells a hop's
 * reductions apart), then the global-timer nanoseconds of the block's
 * arrival, of its start after the wait for the preceding kernel, and of its
 * end. Reduction record: stage << 32 | sums, then eight phase times and the
 * end. NULL, NULL stops the recording. The default build returns
 * WD_ERR_INVALID_ARG. */
int wd_timeline_set(void* blocks, void* phases);

/* Human-readable name of a status code (static string). */
const char* wd_status_string(int status);

/* Text of the last error raised on handle h (static storage owned by h). */
const char* wd_last_error(const wd_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* WD_H */
