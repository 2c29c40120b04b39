/*
 * dmrg_b300.h -- C ABI of the B300 two-site DMRG hot path (arXiv 2311.14106).
 *
 * The library computes sigma = H_eff * psi for the two-site window of ab
 * initio DMRG on the generic Hamiltonian of Eq. 1 (Sec. II.A), builds the
 * renormalized block operators it needs (normal and complementary, Sec. II.A
 * "renormalized block operators"), runs the Davidson diagonalisation
 * (Sec. II.A, "Lanczos or Davidson") and two-site sweeps over an MPS (Eq. 4).
 *
 * Conventions
 *   - All calls return int: DMRG_OK (0) or a negative DMRG_ERR_* code.  No
 *     exception crosses the ABI.  dmrg_last_error(ctx) holds a message.
 *   - Floating point data are IEEE double, row-major, owned by the caller and
 *     copied by the library unless stated otherwise.
 *   - "device pointer" arguments point to CUDA device memory on the current
 *     device; "host pointer" arguments to ordinary host memory.
 *   - stream arguments are cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device work is stream-ordered; calls that return
 *     host scalars synchronise that stream.
 *   - A context is thread-compatible: one thread at a time per context.
 *     Different contexts may be used concurrently.
 *
 * Quantum numbers (QN): spinless model (sym = DMRG_U1) uses (N); spinful
 * (sym = DMRG_U1U1) uses (N_up, N_dn).  Spin-adapted (sym = DMRG_U1SU2,
 * Sec. IV: D counts SU(2) multiplets) uses (N, 2J) for a sector of spin-J
 * multiplets; its sectors are ordered by ((N + 2J)/2, (N - 2J)/2), and all
 * its matrices (isometries, psi) hold reduced elements between multiplets.
 * The site multiplets are {0} (N=0), {up, dn} (N=1, J=1/2, |1/2,+1/2> =
 * c+_up|0>) and {updn} (N=2, J=0, c+_up c+_dn|0>); spins couple in the
 * Jordan-Wigner order of the parts, |(j1 j2) J M> = sum_m <j1 m1 j2 m2|J M>
 * |j1 m1>|j2 m2> (Condon-Shortley), and an enlarged sector's rows run over
 * pieces (site multiplet, block sector) by site multiplet, then block sector.
 * psi pairs L. sector (N_a, 2J) with .R sector (N - N_a, 2J) (total S = 0).
 * Spin-orbital modes along the chain:
 * spinless p = i, spinful p = 2 i (up), 2 i + 1 (down); site i = DMRG site i.
 * Site states are ordered by QN: spinless {0, 1}; spinful
 * {0, dn, up, updn} = QN (0,0), (0,1), (1,0), (1,1), with |updn> =
 * c+_up c+_dn |0>.
 *
 * Isometries (a basis of the MPS, Eq. 4): left isometry n maps the enlarged
 * block L_{n-1} x site_{n-1} onto the block L_n; right isometry n maps
 * site_n x R_{n+1} onto R_n.  For each QN Q of the new block it is a
 * (rows = dim_enlarged(Q)) x (cols = dim_new(Q)) matrix with orthonormal
 * columns.  The rows of an enlarged sector run over pieces ordered by the
 * site state's QN; each piece holds all states of the block sector
 * Q - q(site state), in that sector's order.
 *
 * psi / sigma for window (l, l+1): one block per sector a of L. = L_l x
 * site_l (ascending QN) paired with the sector target - q_a of
 * .R = site_{l+1} x R_{l+2}, stored row-major (dim_a x dim_b), concatenated
 * in that order (dmrg_heff_layout).
 */
#ifndef DMRG_B300_H
#define DMRG_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DMRG_OK = 0,
  DMRG_ERR_ARG = -1,            /* invalid argument or size */
  DMRG_ERR_OOM = -2,            /* device or host allocation failed */
  DMRG_ERR_CUDA = -3,           /* CUDA runtime / cuSOLVER error */
  DMRG_ERR_STATE = -4,          /* call made in the wrong order */
  DMRG_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
  DMRG_ERR_NOT_CONVERGED = -6   /* Davidson hit its iteration limit */
};

enum { DMRG_U1 = 1, DMRG_U1U1 = 2, DMRG_U1SU2 = 3 };   /* symmetry */
enum { DMRG_FP64 = 0, DMRG_SPLIT = 1 };         /* H_eff*psi precision */
enum { DMRG_MODEL_SPINLESS_TV = 1, DMRG_MODEL_HUBBARD = 2 };

typedef struct dmrg_ctx dmrg_ctx;   /* opaque, owned by the library */

typedef struct {
  int sym;                 /* DMRG_U1 (spinless), DMRG_U1U1 (spinful, S_z
                              sectors) or DMRG_U1SU2 (spinful, spin-adapted) */
  int n_sites;             /* N lattice sites = spatial modes */
  int n_up;                /* target particles (spinless: N; U1SU2: all N) */
  int n_dn;                /* target down particles (U1U1 only) */
  int d_max;               /* bond dimension D kept by truncation */
  int precision;           /* DMRG_FP64 or DMRG_SPLIT for H_eff*psi */
  double davidson_tol;     /* residual 2-norm bound, normalized vector */
  int davidson_max_sub;    /* Davidson subspace size (>= 4) */
  int davidson_max_iter;   /* Davidson iteration limit */
  size_t hbm_budget_bytes; /* HBM for renormalized block operators; 0 = no
                              limit (see dmrg_staging_stats) */
  uint64_t seed;           /* seed of the Davidson start vectors */
  int twice_s;             /* U1SU2: twice the total spin S (this build: 0) */
} dmrg_config;

const char *dmrg_error_string(int code);
const char *dmrg_last_error(const dmrg_ctx *ctx);

/* Create a context on the current CUDA device.  cfg is copied.
 * Errors: ARG (bad sizes), CUDA (no device), OOM. */
int dmrg_create(dmrg_ctx **out, const dmrg_config *cfg);
/* Free all device and host memory of ctx.  NULL is accepted. */
int dmrg_destroy(dmrg_ctx *ctx);

/* a1 -- Eq. 2 / Eq. 3 on an Lx x Ly torus (Sec. II.A), site i = y*Lx + x.
 * model DMRG_MODEL_SPINLESS_TV: t (NN), tp (NNN), v = V (NN n_i n_j);
 * model DMRG_MODEL_HUBBARD: t, v = U (on-site), tp ignored.
 * Hopping enters as -t (c+_i c_j + h.c.).  Writes host arrays
 * t_out[N*N] and V_out[N^4] in the Eq. 1 order c+_i c+_j c_k c_l
 * (Hubbard: V[iiii] = U/2 with the spin-independent convention of
 * dmrg_set_hamiltonian).  Requires Lx, Ly >= 3.  Errors: ARG. */
int dmrg_lattice_hamiltonian(int model, int Lx, int Ly, double t, double tp,
                             double v, double *t_out, double *V_out);

/* a2 helper -- real standing-wave momentum modes (Sec. II.B mode basis):
 * U_out[N*N] host, U[i*N + m] = amplitude of mode m on site i, modes ordered
 * by (-2(cos kx + cos ky), nx, ny, cos before sin).  Errors: ARG. */
int dmrg_momentum_basis(int Lx, int Ly, double *U_out);

/* a1/a2 -- Eq. 1 input and the one-particle mode rotation (Sec. II.B):
 * host pointers t[N*N], V[N^4] (Eq. 1 order), U[N*N] orthogonal or NULL
 * (identity).  The library rotates the parameters, t' = U^T t U and
 * V'_abcd = sum V_ijkl U_ia U_jb U_kc U_ld, and forms the spin-orbital
 * antisymmetrised two-body tensor.  Spinful models use the spin-independent
 * form sum_{ab} V_ijkl c+_{ia} c+_{jb} c_{kb} c_{la}.
 * Errors: ARG (NULL, non-orthogonal U, non-Hermitian V: V_ijkl != V_lkji). */
int dmrg_set_hamiltonian(dmrg_ctx *ctx, const double *t, const double *V,
                         const double *U);

/* Eq. 4 -- hand one isometry of the MPS basis to the library (copied).
 * side 0 = left isometry `site` (1..N-1), side 1 = right isometry `site`
 * (1..N-1).  qn[n_sectors * nq] (nq = 1 or 2), rows[], cols[] per sector,
 * data = concatenated row-major matrices (host).  Rows must equal the
 * enlarged sector dimension implied by the previous isometry.
 * Errors: ARG, STATE (isometries out of order), OOM. */
int dmrg_set_isometry(dmrg_ctx *ctx, int side, int site, int n_sectors,
                      const int *qn, const int *rows, const int *cols,
                      const double *data);

/* Eq. 4 -- a seeded random right-canonical MPS basis as the start of
 * dmrg_sweep (the paper's runs start from a warm-up state the configs do not
 * fix): right isometries 1..N-1 made by the library, each sector's columns
 * an orthonormalised Gaussian matrix (splitmix64 / Box-Muller deviates),
 * keeping at most d_max states (multiplets) spread over the sectors in
 * proportion to their dimension (at least one per sector).  Replaces the
 * right isometries set before.  Errors: ARG. */
int dmrg_random_start(dmrg_ctx *ctx, uint64_t seed);

/* a3/a4 -- build the renormalized block operators L_0..L_l and R_N..R_{l+2}
 * from the isometries, the enlarged blocks L. and .R of window (l, l+1) and
 * the sector tables of H_eff (Sec. II.A "Tables").  Errors: STATE, OOM, CUDA. */
int dmrg_build_block_ops(dmrg_ctx *ctx, int l, void *stream);

/* psi layout of the current window: *psi_len elements; *n_blocks blocks;
 * if blocks != NULL it receives 2*nq + 2 ints per block
 * (q_a[nq], q_b[nq], dim_a, dim_b).  Errors: STATE. */
int dmrg_heff_layout(dmrg_ctx *ctx, long long *psi_len, int *n_blocks,
                     int *blocks);

/* Mixed-precision refinement of split-precision Davidson solves (see
 * dmrg_davidson): on windows whose H_eff*psi has at least min_window_flops
 * algorithmic flops, each FP64 refinement step expands its subspace with an
 * approximate solution of the Jacobi-Davidson correction equation
 * (I - u u^T)(H - theta)(I - u u^T) t = -r, from inner_steps preconditioned
 * conjugate-gradient steps with the split-precision product, instead of the
 * diagonally preconditioned residual; the FP64 Rayleigh-Ritz step keeps the
 * result exact to FP64 (fewer FP64 products per solve).  inner_steps = 0
 * turns it off.  Defaults: 20 steps, 1e8 flops.  Errors: ARG. */
int dmrg_set_refinement(dmrg_ctx *ctx, int inner_steps, double min_window_flops);

/* Split-precision contexts solve the windows whose H_eff*psi has fewer than
 * min_window_flops algorithmic flops with the FP64 product alone (Davidson
 * and the energy as in a DMRG_FP64 context); dmrg_heff_apply itself is not
 * affected.  Small windows are launch-bound on both paths, and the split
 * Davidson's noise floor and refinement cost it more products there.
 * Default 0 (every window split).  Errors: ARG. */
int dmrg_set_split_min_flops(dmrg_ctx *ctx, double min_window_flops);

/* Select the arithmetic of dmrg_heff_apply: DMRG_FP64 or DMRG_SPLIT. */
int dmrg_set_precision(dmrg_ctx *ctx, int precision);

/* a5 -- sigma = H_eff * psi (Sec. II.A, Davidson matvec).  psi, sigma:
 * device pointers, psi_len doubles each, owned by the caller; sigma is
 * overwritten; psi is not modified.  Stream-ordered, no host sync.
 * Errors: STATE (no window built), ARG (NULL), TIMEOUT.  A bounded device
 * wait that gave up inside an earlier split-precision call (whose sigma is
 * then incomplete) is reported as TIMEOUT by the first call of this context
 * that runs after the status of that call has reached the host, or by
 * dmrg_sync; it is reported once, and the call that reports it does no work. */
int dmrg_heff_apply(dmrg_ctx *ctx, const double *psi, double *sigma,
                    void *stream);

/* a5, several vectors -- sigma_v = H_eff * psi_v for v = 0..nv-1 (1 <= nv
 * <= 64): psi and sigma are device pointers to nv * psi_len doubles, vector v
 * at v * psi_len.  With DMRG_SPLIT the nv products run in one pass of the
 * split kernels (the batched sector algebra of Sec. III.B): every work item
 * appears once per vector, the copies side by side in the claim order, so an
 * operator tile read from HBM serves all nv vectors from L2.  Each sigma_v is
 * bitwise the result of dmrg_heff_apply on psi_v.  With DMRG_FP64 the
 * vectors are applied one by one.  Stream-ordered; errors as dmrg_heff_apply
 * (ARG for nv out of range). */
int dmrg_heff_apply_batch(dmrg_ctx *ctx, int nv, const double *psi, double *sigma,
                          void *stream);

/* Synchronise `stream` and report the outcome of this context's work on it:
 * DMRG_ERR_TIMEOUT if a bounded device wait of any earlier H_eff*psi of this
 * context (dmrg_heff_apply or dmrg_heff_apply_split_static) gave up and has
 * not been reported yet, else DMRG_OK.  Errors: ARG, CUDA, TIMEOUT. */
int dmrg_sync(dmrg_ctx *ctx, void *stream);

/* Allocation-free variant of dmrg_heff_apply in the split precision
 * (DMRG_SPLIT: FP16 hi + lo operands with per-block power-of-two scales).
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library allocate device memory on the call path (for
 * example code running under another framework's memory pool, or code that
 * must not trigger the implicit synchronisation of cudaMalloc / cudaFree).
 * The per-call scratch of the split path (psi^T in FP16 hi + lo, the stage-1
 * intermediate, the stage-2 partial tiles and the work tables) is taken from
 * a fixed 64 MiB array that every GPU loading this library holds until the
 * process exits; the call itself makes no cudaMalloc, cudaFree or other
 * allocating device call.
 *   - psi, sigma: device pointers as for dmrg_heff_apply; sigma is
 *     overwritten.  The result equals dmrg_heff_apply's split result.
 *   - Needs the window's FP16 operator copies, which the first
 *     dmrg_heff_apply with DMRG_SPLIT creates (Errors: STATE if absent).
 *   - A window whose scratch exceeds 64 MiB is rejected with DMRG_ERR_ARG and
 *     a message giving the size it needs.
 *   - The first call on a device looks up the array's device address, and the
 *     first call for a window writes its work tables into the array; make
 *     that first call before any stream capture.
 *   - All calls (all contexts) share the one array, which keeps the last
 *     call's contents; calls whose GPU work overlaps in time race with each
 *     other and give wrong results.  Serialize them (one stream, or events).
 *   - A bounded device wait that gave up leaves an error word set in the
 *     array; it is cleared only when read.  A later call of the same context
 *     (once the status of the failed call has reached the host) or dmrg_sync
 *     reports it as DMRG_ERR_TIMEOUT, once.
 */
int dmrg_heff_apply_split_static(dmrg_ctx *ctx, const double *psi,
                                double *sigma, void *stream);

/* Same as dmrg_heff_apply but with host buffers: copies psi to the device,
 * applies, copies sigma back, synchronising the stream. */
int dmrg_heff_apply_host(dmrg_ctx *ctx, const double *psi_host,
                         double *sigma_host, void *stream);

/* Algorithmic flops of one H_eff*psi of the current window:
 * sum over nonzero (term, sector) of 2 (m' m n + m' n n'). */
int dmrg_heff_flops(dmrg_ctx *ctx, double *flops);

/* a6 -- lowest eigenpair of H_eff by Davidson (Sec. II.A).  psi_inout:
 * device pointer, start vector on input (need not be normalized; a zero
 * vector means "use a seeded random start"), normalized eigenvector on
 * output.  With DMRG_SPLIT the split product runs until its residual
 * stagnates near its noise floor (about 4e-6 |E|); Davidson iterations with
 * the FP64 product, started from that vector, then take the residual to
 * davidson_tol (mixed-precision refinement; on windows of at least
 * dmrg_set_refinement's flops those iterations expand with a split-precision
 * solution of the correction equation; windows below dmrg_set_split_min_flops
 * are solved with the FP64 product alone).  The energy is the Rayleigh
 * quotient of the FP64 product whatever the precision setting.
 * Errors: STATE, NOT_CONVERGED (psi and energy still written), TIMEOUT. */
int dmrg_davidson(dmrg_ctx *ctx, double *psi_inout, double *energy,
                  int *iters, void *stream);

/* a7 -- truncate the current window's psi (device pointer, normalized) to
 * d_max states (largest Schmidt values over all sectors, ties by lower
 * sector index then lower in-sector index) and renormalize the block on
 * `side` (0: L. -> L_{l+1}, 1: .R -> R_{l+1}).  Outputs discarded weight and
 * entropy (either may be NULL). */
int dmrg_truncate(dmrg_ctx *ctx, const double *psi, int side, int d_max,
                  double *discarded, double *entropy, void *stream);

/* a6-a8 -- two-site sweeps from the right-canonical MPS given by the right
 * isometries.  One sweep = windows l = 0..N-2 left to right (truncating to
 * the left after each window but the last) then l = N-2..0 right to left
 * (truncating to the right after each window but the last).
 * d_schedule[n_sweeps] (NULL = cfg.d_max).  energies_out[n_sweeps] (host)
 * receives the energy of the final window of each sweep.
 * Errors: STATE, OOM, CUDA, TIMEOUT; NOT_CONVERGED if any window's Davidson
 * hit davidson_max_iter (the energies are still written; dmrg_last_error
 * gives the number of such windows). */
int dmrg_sweep(dmrg_ctx *ctx, int n_sweeps, const int *d_schedule,
               double *energies_out, void *stream);

/* Eq. 4 -- read back one isometry of the current MPS basis: after
 * dmrg_sweep, the isometries the sweeps made (left 1..N-2 from the last
 * left-to-right pass, right 2..N-1 from the final right-to-left pass, which
 * with dmrg_get_center give the final state); before any sweep, those set by
 * dmrg_set_isometry.  side 0 = left, 1 = right isometry `site`, in the
 * layout of dmrg_set_isometry.  *n_sectors and *n_elems (sum of rows*cols)
 * are always written; qn[n_sectors*nq], rows[], cols[] and data[n_elems]
 * (host, row-major per sector, concatenated) are filled when not NULL.
 * Errors: ARG (no such isometry). */
int dmrg_get_mps(dmrg_ctx *ctx, int side, int site, int *n_sectors,
                 long long *n_elems, int *qn, int *rows, int *cols,
                 double *data);

/* The normalized two-site center tensor psi of the final window of the last
 * dmrg_sweep (window *l, layout of dmrg_heff_layout for that window):
 * *psi_len always written, psi (host, may be NULL) filled.
 * Errors: STATE (no sweep has run). */
int dmrg_get_center(dmrg_ctx *ctx, int *l, long long *psi_len, double *psi);

/* Work of the two H_eff*psi stages of the current window (for rooflines):
 * out6 = [stage-1 flops, stage-2 flops, A-stack elements, B-stack elements,
 * intermediate T elements, psi_len].  Stage 1 computes T = A psi per term
 * class, stage 2 sigma = sum T B^T; a stored element is 8 bytes on the FP64
 * path and 4 bytes (FP16 hi + lo) on the split path. */
int dmrg_heff_stage_info(dmrg_ctx *ctx, double *out6);

/* Per-kernel timing of dmrg_heff_apply with CUDA events recorded on the
 * apply stream.  enable = 1 starts (and zeroes) the accumulation, 0 stops
 * it.  out5 (may be NULL) receives accumulated milliseconds of
 * [0] psi split (split path), [1] stage 1, [2] stage 2, [3] sum of the
 * split-K partial tiles (split path; the FP64 path sums inside stage 2),
 * and [4] the number of applies timed; reading synchronises the last timed
 * apply. */
int dmrg_heff_timing(dmrg_ctx *ctx, int enable, double *out5);

/* Autotuner record of this context: *n_entries pairs (candidate,
 * milliseconds per split-precision apply) timed on the first window whose
 * operator stacks exceed 256 MB: first the stage-2 split-K ranges (candidate
 * = the range, 1024 / 2048 / 4096), then, with the chosen range, the stage-1
 * schedules (candidate = 100000 + 10 * tile-width cap + item order; caps 128
 * and 64; order 0 rounds from the heavy, light and middle thirds of the
 * cost-sorted items, 1 cost order, 2 heaviest and lightest alternating).  The
 * fastest of each (a later candidate must win by 1.5 %) is used for the rest
 * of the context.  out (may be NULL) receives up to max_entries pairs. */
int dmrg_heff_tuning(dmrg_ctx *ctx, double *out, int max_entries, int *n_entries);

/* Term structure of the window's H_eff: entry i couples input psi block
 * out[3i] to output block out[3i+1] through out[3i+2] operator products (one
 * class of terms with a common quantum-number shift).  Writes at most
 * max_entries triples; *n_entries receives the total (out may be NULL to
 * query it).  DMRG_ERR_STATE without a window. */
int dmrg_heff_entries(dmrg_ctx *ctx, int *out, int max_entries, int *n_entries);

/* Shape of the split-precision plan of the current window (built by the
 * first split apply): out4[0] = kernel launches per apply, [1] stage-1
 * tiles, [2] stage-2 tiles, [3] split-K range of stage 2 (K elements per
 * partial tile).  DMRG_ERR_STATE before the plan exists. */
int dmrg_heff_split_plan(dmrg_ctx *ctx, double *out4);

/* One-particle reduced density matrix (Sec. II.B: gamma_ij = <c+_j c_i>,
 * used for natural orbitals and, back-rotated, for order parameters) of the
 * state psi (device pointer, the current window's layout, normalized by the
 * caller) from the window's block operators: gamma[i*N + j] (host, N*N) =
 * sum over spin of <c+_{j s} c_{i s}> in the rotated mode basis of
 * dmrg_set_hamiltonian (spinless: <c+_j c_i>).  The real-space matrix is
 * U gamma U^T with U the mode rotation.  Synchronises the stream.
 * Errors: ARG, STATE (no window). */
int dmrg_rdm1(dmrg_ctx *ctx, const double *psi, double *gamma, void *stream);

/* Staging of renormalized block operators under cfg.hbm_budget_bytes (the
 * paper's H2D/D2H traffic of operators that do not fit the GPUs, Sec. III.B).
 * With a budget, dmrg_sweep and dmrg_build_block_ops keep at most that many
 * bytes of block operators in HBM (plus the blocks the current window
 * needs): a block the sweep rebuilds before its next use is released, the
 * blocks used last are copied once to pinned host memory and freed on the
 * device, and they come back on a side stream ahead of the window that
 * needs them.  Results are bitwise the same as without a budget.
 * out8: [0] bytes copied host->device, [1] seconds of those copies (CUDA
 * events on the side stream), [2] bytes copied device->host, [3] peak
 * resident block bytes, [4] offloads, [5] reloads, [6] releases, [7] the
 * budget.  Counters accumulate over the context's life.  Errors: ARG. */
int dmrg_staging_stats(dmrg_ctx *ctx, double *out8);

/* Memory of the FP64 path of the current window.  Its operator stacks and
 * its intermediate T sit at fixed device addresses whose physical memory can
 * be given back: T is backed on the first FP64 H_eff*psi, and with
 * cfg.hbm_budget_bytes > 0 the stacks and T are given back as soon as the
 * split path has built its FP16 copies (the next FP64 H_eff*psi gathers the
 * stacks again from the window's blocks, stream-ordered; results are
 * bitwise the same).  out4: [0] 1 if the FP64 stacks are backed, [1] 1 if T
 * is backed, [2] bytes of the stacks, [3] bytes of T.  Errors: ARG, STATE
 * (no window). */
int dmrg_heff_fp64_state(dmrg_ctx *ctx, long long *out4);

/* Windows from sweep position (pass 0 = left to right at window l, pass 1 =
 * right to left) to the next use of block L_n (left = 1) or R_n (left = 0),
 * -1 if the sweep rebuilds it first, -2 for bad arguments: the staging
 * policy, exposed for tests (pure host function, no context). */
long long dmrg_sweep_next_use(int n_sites, int pass, int l, int left, int n);

/* Tile shape and folding the grouped FP64 GEMM picks for `batch` problems of
 * M x N (renormalization products, FP64 H_eff stages): out3 = {tile rows,
 * tile columns, fold} with fold 0 (separate problems), 1 (batch folded into
 * the rows; allowed if fold_rows_ok, i.e. all problems share the B operand)
 * or 2 (into the columns; fold_cols_ok, shared A); square_only restricts the
 * shapes to 16, 32 and 64 squares without folding.  The choice issues the
 * fewest multiply-adds, with a small penalty on small tiles (pure host
 * function, exposed for tests).  Errors: ARG. */
int dmrg_gemm_tile_choice(int M, int N, int batch, int fold_rows_ok, int fold_cols_ok,
                          int square_only, int *out3);

/* Code paths the split-precision plan of the current window exercises
 * (for tests): out8[0] stage-1 work items, [1] stage-2 work items, [2] psi
 * blocks with a side longer than 128 (more than one MMA tile), [3] / [4]
 * stage-2 items packing R = 2 / R = 4 small blocks per tile, [5] largest
 * number of split-K partial tiles of one sigma block, [6] sigma blocks with
 * more than one partial tile, [7] unpacked stage-2 items that are not the
 * first tile of their block.  Errors: STATE before the first split apply. */
int dmrg_heff_split_paths(dmrg_ctx *ctx, long long *out8);

/* Replay the split-precision apply from captured CUDA graphs (default 1), one
 * graph per (psi, sigma) pointer pair; 0 launches the kernels directly. */
int dmrg_set_graphs(dmrg_ctx *ctx, int enable);

/* Self-test of the tcgen05 kernels' bounded waits (no counterpart in the
 * paper): one device thread waits on a shared-memory barrier that nothing
 * completes, with the same wait the H_eff*psi kernels use.  The wait gives up
 * after about one second (2^31 SM cycles) and reports it; nothing faults and
 * the context stays usable.  stream: CUDA stream or NULL.  Returns
 * DMRG_ERR_TIMEOUT when the wait gave up as designed (the expected result),
 * DMRG_ERR_CUDA if it did not or a CUDA call failed, DMRG_ERR_OOM if the
 * 4-byte flag could not be allocated. */
int dmrg_selftest_bounded_wait(void *stream);

/* Self-test of the time-out report (no counterpart in the paper): runs the
 * wait of dmrg_selftest_bounded_wait on this context's error word -- which 0:
 * the window's (needs a split plan), 1: the allocation-free path's -- so that
 * the word is set exactly as a pipeline wait that gave up would set it, and
 * posts it as an H_eff*psi call does.  Nothing faults; the next
 * dmrg_heff_apply / dmrg_heff_apply_split_static / dmrg_sync of the context
 * must then return DMRG_ERR_TIMEOUT once.  Errors: ARG, STATE, CUDA. */
int dmrg_selftest_timeout_report(dmrg_ctx *ctx, int which, void *stream);

/* Timing breakdown of the last sweep in seconds, Sec. III.B categories:
 * out[0] Diag_H, [1] Ren (block ops), [2] Tables, [3] Diag_D, [4] StVec,
 * [5] Other; out[6] = number of H_eff*psi calls. */
int dmrg_profile(dmrg_ctx *ctx, double *out7);

/* Device memory of the context's largest objects so far, in bytes: out6[0]
 * largest renormalized block (operator data), [1] largest enlarged block
 * (block x site, before renormalization, or a window's L. / .R), [2] largest
 * renormalization temporary (the products U_k T_i are computed in chunks of
 * at most 2 GB), [3] FP64 operator stacks of the last window, [4] its split
 * FP16 (hi, lo) copies, [5] the most device memory in use (all processes)
 * seen after a window build.  Errors: ARG. */
int dmrg_memory_stats(dmrg_ctx *ctx, double *out6);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_B300_H */
