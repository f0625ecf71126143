/*
 * libdclno -- the data-parallel hot path of the O(N) divide-conquer method
 * with localized natural orbitals (DC-LNO; Ozaki, Fukuda and Jiang), on one
 * NVIDIA GB300 (sm_103a).
 *
 * One DC-LNO step (Sec. II.C, steps (i)-(v)):
 *   dclno_compute_lnos    LNOs of every atom from its block of the occupied-space
 *                         projector: Lambda_0i = sum_Rj rho_{0i,Rj} S_{Rj,0i}
 *                         (Eq. (Lambda)), V^-1 Lambda V = lambda (Eq. (eigendecomp)),
 *                         keep the leading k eigenvectors (Eq. (apop_Lambda)).
 *   dclno_solve_clusters  for every atom i: H^(i), S^(i) of its truncated cluster in
 *                         the mixed PAO/LNO basis (Eq. (Hi)); H^(i) c = eps S^(i) c;
 *                         central-atom weights of the spectral Green function (Eq. (Gi)).
 *   dclno_find_mu         the common chemical potential that conserves the electron
 *                         count (Sec. II.C step (iv)).
 *   dclno_density_matrix  density-matrix rows of every central atom (Eq. (dm) with
 *                         Eq. (Gi)), kept where S != 0, and the band energy.
 * dclno_build_clusters fixes the truncated clusters (Fig. 1; short-range region of
 * radius r_core with PAOs, long-range region up to r_lno with k LNOs per atom).
 *
 * Conventions (all calls):
 *  - Units: bohr and hartree.  Spin-unpolarised: a factor 2 is applied inside
 *    electron counts and band energies (Sec. II.B, N_ele = 2 tr[rho S]).
 *  - Matrices of the system are block-sparse rows (BSR) keyed by (i, j, R):
 *    row i holds blocks row_ptr[i] .. row_ptr[i+1]-1, sorted by (col, shift[0],
 *    shift[1], shift[2]); block b is the M_i x M_col row-major matrix starting at
 *    element blk_off[b] of a value array.  These are the paper's blocks
 *    S_{0i,Rj}, H_{0i,Rj} of Sec. II.B.  Density matrices use the same pattern.
 *  - Ownership: the caller owns every pointer it passes (host or device as
 *    stated); the context owns its device workspace.  A context keeps pointers
 *    to the caller's device H and S until it is destroyed or rebuilt: they must
 *    stay valid and unchanged in between.
 *  - Streams: all GPU work is ordered on the stream given to dclno_create (NULL =
 *    legacy default stream).  Calls that return host scalars synchronise it.
 *  - Errors: every call returns a dclno_status; on failure dclno_last_error()
 *    gives a message (with the first failing cluster where there is one).  No
 *    call prints or aborts.  A context is single-threaded.
 */
#ifndef DCLNO_H
#define DCLNO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DCLNO_OK = 0,
    DCLNO_ERR_ARG = 1,            /* invalid argument or call order */
    DCLNO_ERR_CUDA = 2,           /* CUDA runtime error */
    DCLNO_ERR_OOM = 3,            /* device workspace could not be allocated */
    DCLNO_ERR_NOT_SPD = 4,        /* a cluster overlap S^(i) is not positive definite */
    DCLNO_ERR_NO_BRACKET = 5,     /* N_e lies outside [N(mu_lo), N(mu_hi)] */
    DCLNO_ERR_NOT_CONVERGED = 6,  /* an eigensolver iteration did not converge */
    DCLNO_ERR_TIMEOUT = 7,        /* a bounded device wait ran out */
    DCLNO_ERR_NO_LNOS = 8         /* solve requested before LNOs were computed */
} dclno_status;

typedef enum {
    DCLNO_FP64 = 0,   /* every step in FP64 */
    DCLNO_MIXED = 1   /* the cubic contractions on BF16 tensor cores, FP64 emulated by
                         8-bit slices (FP64-level accuracy); everything else FP64 */
} dclno_precision;

/* Eigenproblem of the LNOs (dclno_set_lno_mode). */
typedef enum {
    DCLNO_LNO_PAPER = 0,  /* the nonsymmetric Lambda_0i = (rho S)_{0i,0i} of Eq. (Lambda) */
    DCLNO_LNO_SYM = 1     /* the projector form (S rho S)_{0i,0i} v = lambda S_ii v */
} dclno_lno_mode;

/* LNO eigenvalue flags returned by dclno_get_lnos (bit set per atom). */
#define DCLNO_LNO_COMPLEX_SELECTED 1 /* a selected eigenvalue of Lambda is complex */
#define DCLNO_LNO_PAIR_SPLIT 2       /* a complex pair straddles the cut; its real part was kept */

typedef struct dclno_ctx dclno_ctx;

typedef struct {
    int natoms;                /* N */
    const double *pos;         /* host [N][3], atom positions tau_i */
    const double *cell;        /* host [3][3], rows are the lattice vectors */
    const int *pbc;            /* host [3], nonzero = periodic direction */
    const int *norb;           /* host [N], M_i (1 .. 32) */
    long long nnzb;            /* number of stored blocks */
    long long nval;            /* number of stored values (sum of block sizes) */
    const long long *row_ptr;  /* host [N+1] */
    const int *col;            /* host [nnzb] */
    const signed char *shift;  /* host [nnzb][3], cell shift R of each block */
    const long long *blk_off;  /* host [nnzb] */
    const double *H;           /* device [nval], Hamiltonian blocks H_{0i,Rj} */
    const double *S;           /* device [nval], overlap blocks S_{0i,Rj} (symmetric, SPD) */
} dclno_system;

/*
 * Create a context bound to `cuda_stream` (a cudaStream_t, or NULL) on the
 * current CUDA device.  Returns DCLNO_ERR_ARG if out is NULL.
 */
dclno_status dclno_create(dclno_ctx **out, void *cuda_stream);

/* Free the context and its device workspace (NULL is a no-op). */
void dclno_destroy(dclno_ctx *ctx);

/* Message of the last failed call on this context ("" if none); ctx may be NULL. */
const char *dclno_last_error(const dclno_ctx *ctx);

/*
 * Truncated clusters (Fig. 1; Sec. III region construction with fixed radii).
 * For every atom i the cluster holds the images (j, R) with
 * |tau_j + R cell - tau_i| <= r_lno (+1e-9 bohr): those within r_core carry
 * their M_j PAOs, the others k_lno LNOs.  Members are ordered by distance
 * descending, so the central atom is last.  The cluster dimension is
 * n_i = sum_core M_j + k_lno * |LNO members|.  Copies the structure of `sys` to
 * the device, keeps the device pointers sys->H and sys->S, and allocates the
 * solver workspace: for all clusters at once when it fits the budget of
 * dclno_set_workspace_limit, else for the largest of the contiguous batches of
 * clusters that the budget admits (each solved in turn by the calls below).
 * Errors: DCLNO_ERR_ARG (radii, k_lno > M_j, unsorted rows, missing on-site
 * block), DCLNO_ERR_OOM.
 */
dclno_status dclno_build_clusters(dclno_ctx *ctx, const dclno_system *sys,
                                  double r_core, double r_lno, int k_lno);

/*
 * The same with the paper's region rule (Sec. III, steps (i)-(iv)) instead of a
 * fixed short-range radius: for each centre, the images within r_lno are split
 * into first neighbouring atoms (their stored overlap block with the centre has
 * an element of magnitude above s_fna; s_fna = 0 is the literal "non-zero
 * overlap", the centre counts as one) and second neighbouring atoms; the
 * short-range radius is the shell distance whose sphere holds a number of atoms
 * closest to N_F + kappa N_S (ties: the larger sphere), the rest up to r_lno is
 * the long-range (LNO) region.  The paper uses kappa = 3/10.  With Gaussian
 * bases every atom within r_lno overlaps the centre unless s_fna is raised, and
 * the rule then keeps every atom in the short-range region.
 * Errors: as dclno_build_clusters; DCLNO_ERR_ARG for kappa outside [0, 1] or
 * s_fna < 0.
 */
dclno_status dclno_build_clusters_kappa(dclno_ctx *ctx, const dclno_system *sys,
                                        double r_lno, int k_lno, double kappa, double s_fna);

/*
 * LNOs of every atom (Sec. II.B, steps (i)-(iii) of LNO generation):
 * Lambda_0i = sum_Rj rho_{0i,Rj} S_{Rj,0i} (Eq. (Lambda)) from the device density
 * matrix `rho` [nval] in the BSR pattern of S; eigenvalues of the nonsymmetric
 * Lambda_0i by Householder-Hessenberg reduction and Francis double-shift QR;
 * eigenvectors of the k_lno eigenvalues of largest real part by inverse
 * iteration.  The kept vectors are returned to the S_ii-orthonormal basis of
 * their span, each with its largest-magnitude component positive (only the
 * span enters the cluster problem).  A selected complex pair contributes its
 * real and imaginary parts; a pair split by the cut contributes its real part.
 * No-op when k_lno = 0 or r_lno = r_core (rho may then be NULL); otherwise a NULL
 * rho is DCLNO_ERR_ARG.
 */
dclno_status dclno_compute_lnos(dclno_ctx *ctx, const double *rho);

/*
 * Memory admission.  Every cluster needs a private workspace while it is solved
 * and until its density rows are written (about 8 (2.5 n^2 + 40 n) bytes for a
 * cluster of dimension n: H^(i)/A, S^(i)/L, the QL rotation log, strips).
 * dclno_build_clusters splits the clusters (in atom order) into contiguous
 * batches whose workspace fits a budget: `bytes` when set here, otherwise the
 * free device memory left after the context's other arrays, 1 GiB and room for
 * two rho copies.  With one batch nothing changes.  With several, the solve
 * runs batch by batch keeping only eps and q of earlier batches, and the
 * density call solves every batch but the last one again before writing its
 * rows (the same kernels on the same input give the same values), so a step
 * costs up to one extra solve.  Takes effect at the next dclno_build_clusters;
 * 0 restores the automatic budget.  A budget below one cluster's workspace
 * makes dclno_build_clusters fail with DCLNO_ERR_OOM.  The paper has no
 * counterpart (it distributes clusters over MPI ranks, Sec. III).
 */
dclno_status dclno_set_workspace_limit(dclno_ctx *ctx, size_t bytes);

/*
 * After dclno_build_clusters: the number of memory-admitted batches and the
 * bytes of the workspace arena (the largest batch), both host scalars,
 * nullable.
 */
dclno_status dclno_batch_info(dclno_ctx *ctx, int *nbatches_out, size_t *workspace_bytes_out);

/*
 * Launch-shape autotuner (on by default).  The first solve of each batch made
 * outside stream capture (dclno_solve_clusters, dclno_step) times the QL kernel,
 * whose lanes are tridiagonal segments run in lockstep within a warp, at 4, 8, 12,
 * 16, 24 and 32 lanes per warp on the batch's own matrices (restoring its input
 * between tries; the results do not depend on the choice) and keeps the fastest
 * for later solves; this allocates a scratch copy of the batch's tridiagonal
 * matrices once (2 n doubles per cluster).  With it off, or before any eager solve
 * (a first dclno_scf_run), the most lanes that fit in shared memory are used.
 * dclno_get_tuning returns the chosen lanes per warp of batch `batch` (0 = not
 * tuned yet) and, in candidate_ms[6] (host, nullable), the timed milliseconds of
 * each candidate (-1 = not tried).  The paper has no counterpart.
 */
dclno_status dclno_set_autotune(dclno_ctx *ctx, int on);

/*
 * Form of the Householder tridiagonalisation in dclno_solve_clusters (Sec. II.C
 * step (iii); both give the same T up to rounding and the same eigenpairs):
 *   0  automatic (default): the form measured faster on GB300: one-stage in FP64;
 *      in the mixed path two-stage for clusters of dimension >= 128 (torn ones),
 *      one-stage below;
 *   1  one-stage: blocked Householder with a symmetric matrix-vector product per
 *      column (each column reads the whole trailing matrix);
 *   2  two-stage: dense -> band of half-width 32 (blocked Householder whose
 *      products are all matrix-matrix tile products), band -> tridiagonal by
 *      Householder bulge chasing (in double-float arithmetic in the mixed path).
 * The two-stage form keeps a log of about n^2/2 doubles of chase reflectors per
 * cluster, reserved by dclno_build_clusters according to the mode at that time: modes
 * 0 and 2 for clusters of dimension >= 128, mode 1 none.  A
 * cluster uses the two-stage form when the solve allows it (mode 2; mode 0 in the
 * mixed path) and its log exists.  Modes 0 and 1 can be selected at any time, mode 2
 * on a context built in mode 2; each takes effect at the next solve.  Errors:
 * DCLNO_ERR_ARG for another mode, or for mode 2 on clusters built in another mode.
 */
dclno_status dclno_set_tridiag(dclno_ctx *ctx, int mode);

/*
 * Cuppen's tear of the tridiagonal eigenproblem (Sec. II.C step (iii)): clusters of
 * dimension >= 64 are torn at n/2, their two halves solved by implicit QL (a dependent
 * chain of rotations per half) and merged through the secular equation.  Torn twice,
 * each half is torn again at its middle: four QL chains of about a quarter of the
 * rotations each, two merges of halves, then the merge of the halves.  The results
 * are the same eigenpairs up to rounding.
 *   0  automatic (default): twice for clusters of dimension >= 512, once below;
 *   1  once;
 *   2  twice for every torn cluster (dimension >= 64).
 * The segments' rotation logs and the merge matrices are laid out by
 * dclno_build_clusters for the mode selected then (a cluster torn twice holds merge
 * matrices of 4 n ld doubles instead of 2 n ld); selecting another mode after the
 * build returns DCLNO_ERR_ARG, and so does a mode outside 0..2.
 */
dclno_status dclno_set_tear(dclno_ctx *ctx, int mode);

/*
 * Tensor-core engine of the mixed path's emulated FP64 tile products (the same
 * arithmetic and the same bits either way: eight 8-bit slices per FP64 row, exact
 * FP32 level sums, exact 64-bit level combination) for the products with K <= 32
 * (Cholesky, congruence, one-stage tridiagonalisation):
 *   0  chosen per kernel and size bucket by the schedule tuner (default);
 *   1  mma.sync.m16n8k16 BF16 from register fragments;
 *   2  tcgen05.mma with the level accumulators in tensor memory: one thread issues
 *      the products of all eight levels behind one commit, then every warp reads
 *      the levels back (tcgen05.ld) and combines them.
 * The long-K products (Y = A22 V of the band reduction, the merge-matrix products)
 * always run on tcgen05 with one FP64 epilogue per output.  Each CTA using tcgen05
 * holds 256 tensor-memory columns (eight accumulators of 32), at most two such
 * CTAs per SM.  A tensor-core wait that runs out fails the solve
 * with DCLNO_ERR_TIMEOUT (cluster in the message).  Takes effect at the next solve
 * and clears the tuned schedules; DCLNO_ERR_ARG for another value.
 */
dclno_status dclno_set_mixed_engine(dclno_ctx *ctx, int engine);

/*
 * Scheduling of the cubic kernels (Cholesky, congruence, tridiagonalisation, band
 * reduction, bulge chasing).  A batch's clusters, in decreasing-dimension order, form
 * size buckets (dimension rounded up to 64; a bucket below the minimum count of
 * dclno_set_bucket_min merged into its neighbour).  For each bucket and kernel the grid
 * is either one CTA per cluster or persistent (as many CTAs as fit the GPU, each taking
 * clusters from an atomic work counter; no CTA waits on another), and in the mixed
 * path the engine of dclno_set_mixed_engine; consecutive buckets with the same
 * schedule run as one launch.  None of these choices changes a bit of the results.
 * mode 0 (default): the tuner picks: every eager solve of a batch (not one captured
 * into a CUDA graph) times each bucket's kernels under the next untried candidate
 * (timings per cluster, shared by batches with the same rounded dimension), then keeps
 * the fastest, or the untuned default when it is within 2% (at most four solves per
 * precision); 1: one CTA per cluster; 2: persistent.  DCLNO_ERR_ARG for another mode.
 */
dclno_status dclno_set_schedule(dclno_ctx *ctx, int mode);

/*
 * Minimum clusters per size bucket (default 0: twice the GPU's SM count).  Every launch
 * ends in a tail while its last clusters finish, so a bucket of a few clusters costs
 * about the time of one cluster while the rest of the GPU idles; smaller buckets are
 * merged into a neighbour.  1 keeps every 64-wide bucket.  Rebuilds the buckets of the
 * current clusters and clears the tuned schedules; DCLNO_ERR_ARG for a negative count.
 */
dclno_status dclno_set_bucket_min(dclno_ctx *ctx, int count);

/*
 * Text cache of tuned schedules (one line per GPU name, precision, kernel and rounded
 * dimension), read now if the file exists and rewritten whenever the tuner decides a
 * schedule; a later context given the same path starts with those schedules.  NULL
 * switches the cache off.  An unreadable file is treated as empty.
 */
dclno_status dclno_set_tuning_cache(dclno_ctx *ctx, const char *path);

/*
 * JSON summary of the size buckets and their schedules (engine, grid form, whether
 * decided, taken from the cache, and the timed milliseconds of each candidate),
 * written to buf (host, len bytes, NUL-terminated, truncated if short); *needed
 * (nullable) receives the full length including the NUL.
 */
dclno_status dclno_tuning_report(dclno_ctx *ctx, char *buf, size_t len, size_t *needed);
dclno_status dclno_get_tuning(dclno_ctx *ctx, int batch, int *ql_lanes_out, float *candidate_ms);

/*
 * Threshold selection of LNOs (Sec. II.B step (iii)): with on != 0, the next
 * dclno_compute_lnos keeps for each atom the eigenvectors of Lambda whose
 * eigenvalue has a real part >= lambda_th (the paper uses 0.1), at most the
 * k_lno given to dclno_build_clusters (a conjugate pair qualifies as a whole; the
 * cap may split it, as for a fixed count).  Each LNO-region member then carries its
 * own count, so the cluster dimensions change with every LNO computation: the
 * call re-derives them on the host (one synchronisation, no reallocation: the
 * workspace stays laid out for k_lno).  With on = 0 every atom keeps k_lno.
 * dclno_scf_run refuses threshold mode (its steps are captured without host
 * work); loop over dclno_step instead.  dclno_get_lno_counts (host, [N])
 * returns the counts of the last LNO computation (k_lno before any).
 */
dclno_status dclno_set_lno_threshold(dclno_ctx *ctx, int on, double lambda_th);
dclno_status dclno_get_lno_counts(dclno_ctx *ctx, int *counts);

/*
 * Eigenproblem of the next dclno_compute_lnos.  DCLNO_LNO_PAPER (the default) is
 * the paper's nonsymmetric Lambda_0i (Eq. (Lambda), Eq. (eigendecomp)).
 * DCLNO_LNO_SYM takes the same selection from the symmetric-definite projector
 * form: G_i v = lambda S_ii v with G_i = (S rho S)_{0i,0i} =
 * sum_{Ra,Rb} S_{0i,Ra} rho_{Ra,Rb} S_{Rb,0i}, the on-site block of the
 * occupied-space projector in the PAO metric (Sec. II.B); only the symmetric part
 * of G_i enters (the block for (rho + rho^T)/2).  Its eigenvalues are real and lie
 * in [0, 1] when rho is a Fermi projector; the leading k_lno eigenvectors (or
 * those >= lambda_th in threshold mode) are kept, in the same canonical basis.
 * Eigenpairs by Cholesky of S_ii, congruence and cyclic Jacobi.  G_i costs
 * |row i| x |row a| block products per atom (about the square of the neighbour
 * count: far more than Lambda_0i).  Row i's block keys are held in shared memory:
 * a row longer than about 24,000 blocks is refused (DCLNO_ERR_ARG) at
 * dclno_compute_lnos.  An S_ii that is not positive definite fails with
 * DCLNO_ERR_NOT_SPD (atom in the message).  Errors: DCLNO_ERR_ARG for another
 * mode value.
 */
dclno_status dclno_set_lno_mode(dclno_ctx *ctx, dclno_lno_mode mode);

/*
 * Assemble and solve every cluster (Sec. II.C steps (ii)-(iii)): Cholesky
 * S^(i) = L L^T, A = L^-1 H^(i) L^-T, Householder tridiagonalisation A = Q T Q^T
 * (one stage, or dense -> band -> tridiagonal: dclno_set_tridiag), T = Z Theta Z^T
 * by Cuppen's divide and conquer (T torn at n/2, or twice from dimension 512:
 * dclno_set_tear; implicit QL on the segments, merges through the secular
 * equation), and the central-atom rows of the eigenvectors C = L^-T Q Z.  In
 * DCLNO_MIXED the cubic contractions run as emulated FP64 on BF16 tensor cores
 * (dclno_set_mixed_engine) and the two-stage form's bulge chasing in double-float
 * arithmetic on the FP32 pipe; QL, merges and everything after stay FP64.  Keeps per cluster the eigenvalues eps_mu,
 * the weights q_mu = sum_{alpha in i} C_{alpha mu} (S^(i) C)_{alpha mu}
 * (sum_mu q_mu = M_i) and what dclno_density_matrix needs.
 * Errors: DCLNO_ERR_NO_LNOS, DCLNO_ERR_NOT_SPD, DCLNO_ERR_NOT_CONVERGED (cluster id
 * in the message), DCLNO_ERR_ARG for an unsupported precision.
 */
dclno_status dclno_solve_clusters(dclno_ctx *ctx, dclno_precision precision);

/*
 * Common chemical potential (Sec. II.C step (iv)): mu with
 * N(mu) = 2 sum_i sum_mu f((eps_mu^(i) - mu)/kT) q_mu^(i) = n_electrons,
 * f(x) = 1/(1+e^x), by device-wide k-section of [min eps - 40 kT, max eps + 40 kT]
 * to double precision (or |N - N_e| <= 1e-12 N_e).  Writes host scalars
 * mu_out and nelec_out (= N(mu)); either may be NULL.
 * Errors: DCLNO_ERR_NO_BRACKET, DCLNO_ERR_ARG (kT <= 0, no solve yet).
 */
dclno_status dclno_find_mu(dclno_ctx *ctx, double n_electrons, double kT,
                           double *mu_out, double *nelec_out);

/*
 * Density-matrix rows of every central atom at chemical potential mu
 * (Eq. (dm) with the spectral Green function of Eq. (Gi)):
 * rho_{0i alpha, Rj beta} = sum_mu f(eps_mu) c_{mu,0i alpha} c_{mu,Rj beta},
 * with LNO columns returned to PAOs through V_j, written to the device array
 * rho_out [nval] in the BSR pattern of S (zero for pairs outside the cluster).
 * eband_out (host, nullable) = 2 sum_i sum_mu f(eps_mu) eps_mu q_mu.
 */
dclno_status dclno_density_matrix(dclno_ctx *ctx, double mu, double kT,
                                  double *rho_out, double *eband_out);

/*
 * Density matrix and energy density matrix rows together (Sec. II.C step (v)):
 * rho as in dclno_density_matrix, and e_{0i alpha, Rj beta} =
 * sum_mu f(eps_mu) eps_mu c_{mu,0i alpha} c_{mu,Rj beta} (Eq. (edm) with Eq. (Gi))
 * into the device array edm_out [nval] (nullable: then rho only).  The energy
 * density matrix needs M_i <= 16.  2 Tr(e S) equals the band energy.
 */
dclno_status dclno_density_matrices(dclno_ctx *ctx, double mu, double kT,
                                    double *rho_out, double *edm_out, double *eband_out);

/*
 * Density-matrix rows of every central atom from the Green function summed over
 * the Matsubara poles (the paper's Appendix, Eq. (rho0j), in a non-orthogonal
 * basis): rho^(i) = S^-1/2 + (2/beta) Re sum_{p>=0} (z_p S^(i) - H^(i))^-1 with
 * z_p = mu + i (2p+1) pi kT, the same quantity as Eq. (dm) with Eq. (Gi) but without
 * eigenvectors.  Each cluster is reduced as by dclno_solve_clusters (Cholesky,
 * congruence, Householder tridiagonalisation T, in `precision`), then the first
 * n_poles poles cost complex tridiagonal solves with T, and the poles beyond are
 * summed from the large-|z| expansion of (z - T)^-1 to third order with Hurwitz
 * zeta sums.  The rows go to the device array rho_out [nval] in the BSR pattern of
 * S (zero outside the cluster, LNO columns returned to PAOs), as from
 * dclno_density_matrix.  The expansion holds only when the first omitted pole lies
 * well above the cluster's spectrum about mu: a cluster whose Gershgorin bound of
 * |T - mu| exceeds (2 n_poles + 1) pi kT / 3 fails with DCLNO_ERR_ARG (cluster in
 * the message).  Practical for narrow spectra only (the count grows with the
 * spectral width over kT).  Needs LNOs (dclno_compute_lnos); overwrites the
 * workspace of an earlier solve (call dclno_solve_clusters again before
 * dclno_find_mu or dclno_density_matrix).  Allocates a scratch of
 * 2 x 32 x 16 bytes per cluster, row and central basis function of a batch.
 */
dclno_status dclno_density_matrix_poles(dclno_ctx *ctx, double mu, double kT, int n_poles,
                                        dclno_precision precision, double *rho_out);

/*
 * One whole DC-LNO step: compute_lnos(rho_in), solve_clusters(precision),
 * find_mu, density_matrix(rho_out).  With host_buffers != 0, rho_in and rho_out
 * are host arrays [nval] copied to and from the context's device buffers inside
 * the call; otherwise they are device arrays.  rho_in may be NULL where
 * dclno_compute_lnos allows it (no LNO region).  mu_out, nelec_out, eband_out are
 * host scalars (nullable).
 */
dclno_status dclno_step(dclno_ctx *ctx, const double *rho_in, double *rho_out,
                        int host_buffers, dclno_precision precision,
                        double n_electrons, double kT,
                        double *mu_out, double *nelec_out, double *eband_out);

/*
 * Ogita-Aishima refinement of approximate generalised eigendecompositions with
 * FP64 residuals (Ogita & Aishima, Japan J. Indust. Appl. Math. 35 (2018), every
 * inner product taken in the S metric).  Not a step of the paper: the refinement a
 * mixed-precision eigensolver would apply to FP32 eigenpairs.  The library's own
 * mixed path does not call it: at the workloads' conditioning its FP32 start lies
 * outside the region where the sweeps converge, and the emulated FP64 contractions
 * reach FP64 accuracy directly.  For each of `count` independent pencils of
 * dimension n, nsweeps times:
 *   R = I - X^T S X,  G = X^T H X,  lam_i = G_ii / (1 - R_ii),
 *   delta = 2 (||G - diag(lam)||_F + max|lam| ||R||_F),
 *   E_ij = (G_ij + lam_j R_ij) / (lam_j - lam_i) for i != j with |lam_j - lam_i| > delta,
 *   E_ij = R_ij / 2 otherwise,   X <- X + X E.
 * Each sweep squares the error of eigenpairs whose error is below the gaps of
 * their eigenvalues; pairs closer than delta only keep their S-orthonormalisation.
 * H, S: device [count][n][n] (row-major, symmetric, S positive definite); X: device
 * [count][n][n] (in/out, column mu the approximate eigenvector of eigenvalue mu);
 * lam_out: device [count][n], the eigenvalue estimates of the last sweep (from that
 * sweep's input X).  All FP64, contiguous, on the current device; X and lam_out
 * must not overlap each other, H or S.  Costs 10 n^3
 * FP64 flops per pencil and sweep; allocates a workspace of 3 count n^2 + count
 * doubles for the call and synchronises `cuda_stream` (NULL = legacy default
 * stream) before returning.  Errors: DCLNO_ERR_ARG (NULL pointers, n, count or
 * nsweeps < 1, n > 2,097,120 or count > 65,535), DCLNO_ERR_OOM, DCLNO_ERR_CUDA (X is
 * then partly updated).
 */
dclno_status dclno_refine_eigenpairs(const double *H, const double *S, double *X, double *lam_out,
                                     int n, int count, int nsweeps, void *cuda_stream);

/*
 * The chemical-potential search of dclno_find_mu without any device
 * allocation, for callers that cannot call cudaMalloc: applications whose own
 * pool allocator has taken all device memory up front, and control loops that
 * must not allocate once they are running (an allocation can block, fail or
 * fragment memory at a bad moment).  The paper has no counterpart: this is an
 * interface for such callers.
 * Inputs: eps, q: device arrays of `count` eigenvalue / weight pairs (for
 * example a copy of dclno_get_spectrum's output), both contiguous FP64, both
 * holding at least `count` elements, on the device that is current for the
 * calling thread; the library cannot check any of this and reads past a
 * shorter array.  n_electrons, kT as in dclno_find_mu.  Outputs: mu_out,
 * nelec_out (host scalars, nullable), copied to the host at the end of the
 * call.  Work is ordered on `cuda_stream` (NULL = legacy default stream); the
 * call synchronises it.
 * Scratch: a file-scope device array of about 165 KB inside the library,
 * allocated on every GPU that loads the library and kept until exit; it
 * covers at most 8,388,608 pairs (4096 blocks x 256 threads x 8), and a larger
 * count returns DCLNO_ERR_ARG without touching the GPU.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) once and
 * keeps it; make that first call on each device before any stream capture
 * begins there.  All calls share the one array:
 * calls whose GPU work overlaps (other threads or streams) race and must be
 * serialised by the caller.
 * Errors: DCLNO_ERR_ARG (null pointers, count < 1 or too large, kT <= 0),
 * DCLNO_ERR_NO_BRACKET, DCLNO_ERR_CUDA.  No context: there is no message.
 */
dclno_status dclno_find_mu_noalloc(const double *eps, const double *q, long long count,
                                   double n_electrons, double kT, double *mu_out,
                                   double *nelec_out, void *cuda_stream);

/*
 * Self-consistency loop with linear density mixing (Sec. II.C: LNOs are updated
 * every SCF step; H and S are held fixed here): nsteps times
 *   rho_out = DC-LNO step(rho);  rho <- rho + alpha (rho_out - rho)
 * on the device array rho [nval] (in/out).  No host synchronisation inside the
 * loop: statuses, mu and the band energy stay on the device and are checked
 * after it.  With use_graph != 0 one step is captured into a CUDA graph and
 * replayed nsteps times (the context must use a non-default stream).
 * mu_hist, nelec_hist, eband_hist: host arrays [nsteps] (nullable) of mu,
 * N(mu) and E_band per step.  After the call the spectrum of the last step is
 * available through dclno_get_spectrum.
 */
dclno_status dclno_scf_run(dclno_ctx *ctx, double *rho, int nsteps, double alpha,
                           dclno_precision precision, double n_electrons, double kT,
                           int use_graph, double *mu_hist, double *nelec_hist,
                           double *eband_hist);

/* ---- inspection (tests, benchmarks) ------------------------------------ */

/*
 * Cluster sizes after dclno_build_clusters: dims_out [N] (host, n_i),
 * nmembers_out [N] (host, members incl. the centre), both nullable.
 * total_out (host, nullable) = sum_i n_i.
 */
dclno_status dclno_cluster_info(dclno_ctx *ctx, int *dims_out, int *nmembers_out,
                                long long *total_out);

/*
 * Spectra after dclno_solve_clusters, cluster by cluster in atom order, each
 * cluster's n_i eigenvalues in solver order (not sorted): eps_out, q_out are
 * host arrays of length sum_i n_i (nullable).
 */
dclno_status dclno_get_spectrum(dclno_ctx *ctx, double *eps_out, double *q_out);

/*
 * LNOs after dclno_compute_lnos, atom by atom: V_out [sum_i M_i k] (host, the
 * M_i x k block of atom i row-major), lam_re/lam_im [sum_i M_i] (host, Lambda
 * eigenvalues sorted by real part descending; in DCLNO_LNO_SYM mode the
 * eigenvalues of G_i v = lambda S_ii v, imaginary parts 0), flags [N] (host).
 * All nullable.
 */
dclno_status dclno_get_lnos(dclno_ctx *ctx, double *V_out, double *lam_re,
                            double *lam_im, int *flags);

/* Number of kernel launches this context has issued so far (for reports). */
long long dclno_launch_count(const dclno_ctx *ctx);

/*
 * Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch (off by default).  dclno_set_profiling(ctx, on) clears the
 * totals and switches recording on or off.  dclno_kernel_time(ctx, name, ...)
 * waits for the recorded launches of kernel `name` (e.g. "k_tridiag") and
 * returns their summed duration in milliseconds and their count (host
 * scalars, nullable); unknown names give 0.
 */
dclno_status dclno_set_profiling(dclno_ctx *ctx, int on);

/*
 * FP64 throughput of the current device, measured in the call with two short
 * kernels (about 0.1 s): FP64 fused multiply-add and FP64 tensor-core MMA
 * (mma.sync m8n8k4), in TFLOP/s (host scalars, nullable).  Used as the
 * denominators of roofline fractions; allocates and frees a small buffer.
 */
dclno_status dclno_measure_fp64_peaks(double *dfma_tflops, double *dmma_tflops);
dclno_status dclno_kernel_time(dclno_ctx *ctx, const char *name, double *total_ms, long long *launches);

#ifdef __cplusplus
}
#endif
#endif /* DCLNO_H */
