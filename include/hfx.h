/*
 * libhfx -- screened, linear-scaling periodic Hartree-Fock exchange build under
 * localized resolution of the identity (LRI), for one NVIDIA GB300 (sm_103a).
 *
 * Method: Lin, Ren and He, arXiv:2009.12505 (linear-scaling periodic exchange
 * with numerical atomic orbitals and LRI).  The library computes
 *
 *   Sigma_{Ii,Jj} = - sum_{K,L} sum_{k,l} sum_{A in {I,K}} sum_{B in {J,L}}
 *                     sum_{alpha,beta} C^{A alpha}_{Ii,Kk} V_{A alpha,B beta}
 *                     C^{B beta}_{Jj,Ll} D_{Kk,Ll}                (Eq. HFX_LRI)
 *
 * built in the <A,B>-pair loop of Algorithm 2/3 with the C((VC)D)
 * multiplication order (Appendix A), screened per term by block upper limits
 * (Sec. III.B/III.C), and E_X = 1/2 sum D . Sigma (Algorithm 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Sites.  A site is (atom a in [0, natoms), lattice vector n in Z^3) (Eq. AO).
 * Block keys are (i, j, n1, n2, n3): the block between site (i, 0) and site
 * (j, n).  |n_k| <= 127.
 *
 * Block shapes, row-major FP64:
 *   C key (a, f, n): [nabf(a)][nao(a)][nao(f)]  -- ABFs on a (Eq. LRI)
 *   V key (a, b, n): [nabf(a)][nabf(b)]         -- (P_a alpha | P_b beta)
 *   D key (k, l, n): [nao(k)][nao(l)]           -- real-space density matrix
 *   Sigma key (i, j, n): [nao(i)][nao(j)]       -- exchange matrix, Ha
 * A block exists iff it was set; the library never infers symmetric partners
 * and never recomputes distances.  Setting a key again replaces it.
 *
 * Screening.  A term (A, B, F, G, variant) survives iff
 *   S = (max|C_AF| * max|C_BG|) * (max|V_AB| * max|D_src|) > theta,
 * multiplied in exactly that association in round-to-nearest FP64, where D_src
 * is the density block the variant contracts with (D_FG, D_FB, D_AG or D_AB).
 * When F is the same site as A (or G as B) the pieces with ABFs on F (or G)
 * are the same term as the ABF-on-A (B) piece and are not added again.
 * The Sigma key set is exactly the keys receiving at least one surviving term.
 *
 * Precision modes (hfx_prec):
 *   HFX_FP64   -- every contraction in FP64 on CUDA cores;
 *   HFX_BF16X3 -- tensor-core contractions with every operand row split into
 *                 two balanced 7-bit digits (exact in BF16) under one
 *                 power-of-two exponent, and only the three leading digit
 *                 products hi*hi, hi*lo, lo*hi formed (about 13 significant
 *                 bits; does not meet 1e-8 Ha, kept for comparison);
 *   HFX_OZAKI  -- the same with nslices digits (4..6) and every digit product
 *                 of order <= nslices - 1: each order's f32 tensor-core sum is
 *                 exact; the orders are added in int64 where a product goes
 *                 straight to Sigma, and in double-float (f32 pairs, rounding
 *                 below the digit truncation) where it feeds a further
 *                 contraction (6 digits: about 41 significant bits per operand
 *                 row).
 * Sigma is accumulated in 128-bit fixed point (integer adds, 2^-64 Ha
 * resolution) and converted to FP64 once, and E_X is summed from it in a
 * fixed order, so results are bitwise reproducible run to run in every mode.
 * Range: every partial contribution a kernel adds, and every finished Sigma
 * element, must stay below 2^31 Ha in magnitude; a kernel that meets a larger
 * contribution adds nothing and the build returns HFX_E_CUDA ("reported
 * error 8").
 *
 * Ownership.  hfx_set_* copy the caller's data (host pointers) or read device
 * pointers on the context's stream before returning; the caller may free or
 * reuse its buffers afterwards.  The context owns all device memory it
 * allocates.  Outputs go to caller buffers.  A context is used by one host
 * thread at a time.
 *
 * Errors.  Every call returns a status and never aborts, traps or exits.
 * hfx_last_error() gives a message for the last failing call on a context.
 * Device-side waits are bounded; expiry returns HFX_E_TIMEOUT.
 */
#ifndef HFX_H
#define HFX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hfx_ctx hfx_ctx;

typedef enum {
  HFX_OK = 0,
  HFX_E_ARG = 1,      /* bad argument: null pointer, out-of-range index, NaN/Inf data */
  HFX_E_SHAPE = 2,    /* sizes inconsistent with nao/nabf */
  HFX_E_STATE = 3,    /* call out of order (e.g. results requested before a build) */
  HFX_E_NOMEM = 4,    /* host or device allocation failed */
  HFX_E_CUDA = 5,     /* a CUDA runtime call or kernel failed */
  HFX_E_TIMEOUT = 6,  /* a bounded device wait expired */
  HFX_E_NOTFOUND = 7  /* key not present */
} hfx_status;

typedef enum { HFX_FP64 = 0, HFX_BF16X3 = 1, HFX_OZAKI = 2 } hfx_prec;

/*
 * Create a context for one periodic system (Sec. II, Eq. AO).
 *   lattice   9 doubles, rows a1, a2, a3 in bohr (recorded; not used to infer blocks)
 *   natoms    number of atoms in the unit cell, >= 1
 *   pos       natoms x 3 Cartesian positions in bohr (recorded), may be NULL
 *   species   natoms species indices in [0, nspecies)
 *   nao/nabf  nspecies NAO and ABF counts per species, 1..64 NAOs, 1..256 ABFs
 *   cuda_stream  cudaStream_t all device work is ordered on; NULL = legacy default
 *   out       receives the context
 * Errors: HFX_E_ARG, HFX_E_NOMEM, HFX_E_CUDA (no usable sm_103 device).
 */
hfx_status hfx_create(const double lattice[9], int32_t natoms, const double *pos,
                      const int32_t *species, int32_t nspecies, const int32_t *nao,
                      const int32_t *nabf, void *cuda_stream, hfx_ctx **out);

/*
 * Set one LRI coefficient block C(a, f, n) (Eq. LRI; Sec. III.B "supermatrix
 * C_{A,F} of dense rank-3 blocks").  blk: [nabf(a)][nao(a)][nao(f)] host FP64.
 * Errors: HFX_E_ARG (index, NaN/Inf), HFX_E_NOMEM.
 */
hfx_status hfx_set_C(hfx_ctx *ctx, int32_t a, int32_t f, const int32_t n[3], const double *blk);

/* Set one Coulomb block V(a, b, n) = (P_a | P_b) (Sec. III.B.2); [nabf(a)][nabf(b)]. */
hfx_status hfx_set_V(hfx_ctx *ctx, int32_t a, int32_t b, const int32_t n[3], const double *blk);

/* Set one density-matrix block D(k, l, n) (Eq. DM_realspace); [nao(k)][nao(l)]. */
hfx_status hfx_set_D(hfx_ctx *ctx, int32_t k, int32_t l, const int32_t n[3], const double *blk);

/*
 * Bulk form of hfx_set_C/V/D.  which: 'C', 'V' or 'D'.
 *   keys  nblk x 5 int32 (i, j, n1, n2, n3), HOST memory
 *   data  packed blocks, block e at data[offs[e] .. offs[e+1]); host or device
 *   offs  nblk + 1 int64 offsets in doubles, HOST memory; offs[e+1]-offs[e]
 *         must equal the block's shape
 *   on_device  0: data is host memory; 1: data is device memory on this GPU
 * Replaces any existing blocks with the same keys.  A call that sets every
 * block of the kind again, in ascending key order (the packed order: keys
 * compared as (i, j, n1, n2, n3)) with the same offsets as the kind's packed
 * blocks after a build, copies the data into the device array in place; any
 * other call copies it into a new device chunk that the next build packs.
 * Errors: HFX_E_ARG, HFX_E_SHAPE, HFX_E_NOMEM, HFX_E_CUDA (after a failed
 * in-place copy the kind's values are undefined until set again).
 */
hfx_status hfx_set_many(hfx_ctx *ctx, char which, int64_t nblk, const int32_t *keys,
                        const double *data, const int64_t *offs, int on_device);

/* Remove every block of one kind ('C', 'V', 'D'). */
hfx_status hfx_clear(hfx_ctx *ctx, char which);

/*
 * Build Sigma and E_X (Algorithm 5 "Calculate exact-exchange": screen, then
 * the staged C((VC)D) contractions of Algorithm 3, then E_X).
 *   theta    screening threshold (>= 0; 0 keeps every term with non-zero blocks)
 *   prec     contraction precision (see above)
 *   nslices  digits per operand: HFX_OZAKI 4..6 (0 = 6), HFX_BF16X3 0 or 2,
 *            HFX_FP64 ignored
 *   ex_out   receives E_X in Ha (host pointer), may be NULL
 * Errors: HFX_E_STATE (no C, V or D set), HFX_E_ARG (also: a split mode with
 *         an atom of more than 32 NAOs), HFX_E_NOMEM, HFX_E_CUDA, HFX_E_TIMEOUT.
 */
hfx_status hfx_build(hfx_ctx *ctx, double theta, hfx_prec prec, int32_t nslices, double *ex_out);

/*
 * Shard the contraction over central atoms (Sec. III.D: pairs <A,B> are
 * distributed over processes; here every pair of central atom A goes to
 * owner[A]).  owner: natoms ranks (host memory, copied); rank: this
 * context's rank.  NULL owner removes the shard.  The screen and the Sigma
 * key set stay global; hfx_build then adds only this rank's terms, and the
 * ranks' fixed-point accumulators (hfx_get_H_fixed) summed elementwise as
 * 64-bit integers equal, bit for bit, those of an unsharded build.
 * Errors: HFX_E_ARG (rank or owner out of range).
 */
hfx_status hfx_set_shard(hfx_ctx *ctx, const int32_t *owner, int32_t rank);

/*
 * The last build's Sigma accumulators: two int64 words per element (units of
 * 2^-32 and 2^-64; element value = w0 2^-32 + w1 2^-64), elements in the
 * hfx_get_H_all layout.  on_device as in hfx_get_H_all.
 */
hfx_status hfx_get_H_fixed(const hfx_ctx *ctx, int64_t *words, int on_device);

/*
 * Replace the last build's accumulators by words (e.g. the elementwise sum
 * over ranks of hfx_get_H_fixed) and recompute Sigma and E_X from them;
 * ex_out (nullable) receives E_X.  The key set must be the last build's.
 */
hfx_status hfx_set_H_fixed(hfx_ctx *ctx, const int64_t *words, int on_device, double *ex_out);

/* Number of Sigma blocks of the last build.  HFX_E_STATE if inputs changed since. */
hfx_status hfx_H_count(const hfx_ctx *ctx, int64_t *nblk);

/* Sigma keys of the last build, nblk x 5 int32, sorted by (i, j, n1, n2, n3). */
hfx_status hfx_H_keys(const hfx_ctx *ctx, int32_t *keys);

/* Offsets (nblk + 1 int64, in doubles) of the blocks in hfx_get_H_all's layout. */
hfx_status hfx_H_offsets(const hfx_ctx *ctx, int64_t *offs);

/*
 * One Sigma block (i, j, n) of the last build into out[nao(i)][nao(j)] (host).
 * Errors: HFX_E_STATE, HFX_E_NOTFOUND (key not in the Sigma key set).
 */
hfx_status hfx_get_H(const hfx_ctx *ctx, int32_t i, int32_t j, const int32_t n[3], double *out);

/*
 * Every Sigma block, packed in key order at hfx_H_offsets, into out.
 * on_device 0: out is host memory; 1: device memory on this GPU.
 */
hfx_status hfx_get_H_all(const hfx_ctx *ctx, double *out, int on_device);

/*
 * Adjoint of the last build with its surviving-term set frozen:
 *   dC receives dE_X/dC packed like the C blocks in key-sorted order
 *   dV receives dE_X/dV packed like the V blocks in key-sorted order
 * (host pointers; either may be NULL).  HFX_E_STATE before a build.
 */
hfx_status hfx_grad(hfx_ctx *ctx, double *dC, double *dV);

/*
 * Build many independent cells (contexts) together, cell c with theta
 * thetas[c] (spec batching; the paper builds one system at a time).
 * The cells are merged into one system -- cell c's atoms follow those of the
 * cells before it, its blocks keep their keys with both atoms offset, no
 * block joins two cells -- and built once: one screen launch and, per wave,
 * one launch of each persistent kernel serve the jobs of every cell, uneven
 * block sizes included.  The screen uses each central atom's own cell's
 * theta.  Each cell then receives its Sigma blocks, its fixed-point words and
 * its E_X (ex_out[c] if ex_out is not NULL), bitwise equal to hfx_build of
 * that cell alone when the cells agree on whether their V and D are exactly
 * Hermitian (the mirror pieces are used for all cells or for none).
 * The cells' input blocks are copied into the merged system, so the device
 * needs room for them twice.  cells[0] keeps the merged system (freed with
 * it): a later batch of the same cells in the same order, in which no cell's
 * C or V blocks and no cell's D key set changed, reuses its plan and sliced
 * operands and copies in only the D blocks that changed (the cached-plan path
 * of an SCF iteration).  Runs on cells[0]'s stream; cells must be distinct
 * and use the same ERI-screen threshold; shards are ignored.
 * After a batch, hfx_get_H*, hfx_H_*, hfx_get_H_fixed, hfx_sigma_k and
 * hfx_stats (batch-wide figures) work on each cell; hfx_grad and
 * hfx_set_H_fixed need a build of the cell alone and return HFX_E_STATE.
 * Errors: HFX_E_ARG (NULL arrays, ncells < 0, a repeated cell, a bad theta,
 * different ERI thresholds), HFX_E_SHAPE (more than 2^20 atoms in all),
 * else the merged build's status, with its message in every cell's
 * hfx_last_error; no cell then holds results.
 */
hfx_status hfx_build_batch(hfx_ctx **cells, int32_t ncells, const double *thetas, hfx_prec prec,
                           int32_t nslices, double *ex_out);

/*
 * Cauchy-Schwarz ERI screen (Sec. III.C, Eq. CS-ERI), applied by the next
 * builds on top of the block screen at theta.  For every C block (x, y, n)
 * the library computes, in FP64 on the GPU, Q = the largest diagonal ERI
 * (phi_Xa phi_Yf | phi_Xa phi_Yf) over the AO pairs of the sites X = (x, 0),
 * Y = (y, n), with the pair expanded by Eq. LRI on the ABFs of X
 * (C(x,y,n)[:, a, f]) and, when Y is another site, of Y (C(y,x,-n)[:, f, a]),
 * using the V blocks between X and Y (missing blocks count as zero).  A
 * quadruple (A, B, F, G) -- AO pairs {A, F} and {B, G} -- keeps its terms only
 * if sqrt(max(Q_AF, 0)) * sqrt(max(Q_BG, 0)) > eps_eri (strict, round-to-
 * nearest FP64).  The bounds are computed once per change of C or V.
 *   eps_eri   threshold in Ha; a negative value turns the screen off (the
 *             default for a new context)
 * Errors: HFX_E_ARG (NULL ctx, NaN or infinite eps_eri).  Marks results stale.
 */
hfx_status hfx_set_eri_screen(hfx_ctx *ctx, double eps_eri);

/* Statistics of the last build (layout: struct hfx_stats_v1 below). */
typedef struct {
  int32_t version;          /* 1 */
  int32_t prec;
  double theta;
  int64_t n_sigma_blocks;
  int64_t n_work_items;     /* <A,B> pairs */
  int64_t n_active_abg;     /* (A,B,G) triples with >= 1 surviving term */
  int64_t survivors[4];     /* surviving terms per variant: ABFs on (I,J),(I,L),(K,J),(K,L) */
  double canonical_flops;   /* Algorithm 3 count: 2 nP(A)nP(B)nao(B)nao(G) per active (A,B,G)
                               + 4 nP(A) x (product of the three AO sizes) per surviving term */
  double executed_flops;    /* multiply-adds x 2 actually issued by this build's kernels */
  double ms_screen, ms_contract, ms_reduce, ms_total;
  int64_t n_waves;
  int64_t scratch_bytes;
  /* per kernel, summed over waves, CUDA events on the context's stream:
     [0] screen, [1] Y = V C, [2] D-stage (P, T3), [3] Q = C D, [4] D_FG piece,
     [5] D_AG piece, [6] D_FB piece, [7] D_AB piece */
  double kernel_ms[8];
  double kernel_flops[8];   /* multiply-adds x 2 issued by each kernel */
  int64_t n_launches;       /* kernels this build launched */
  int32_t mirror;           /* 1: V and D were exactly Hermitian and the mirror pieces were used */
  int32_t nslices;          /* digits per operand in the split modes, else 0 */
  double kernel_tensor_flops[8]; /* bf16 tensor-core flops issued per kernel (split modes) */
  double canonical_flops_piece[4]; /* canonical_flops split by piece (T and Ht stages) ... */
  double canonical_flops_y;        /* ... and the Y = V C part; the five sum to canonical_flops */
  /* split modes: FP64-equivalent flops (2 per multiply-add of the unsplit
     operands) of each tensor-core product, without row, column or K padding
     and without zero tiles; [1] Y, [4] D_FG + D_FB products, else 0 */
  double kernel_unpadded_flops[8];
  /* split modes with tensor-core D_FG / D_FB products: load balance of those
     persistent launches, sum over waves of the largest CTA busy time over the
     sum of the mean CTA busy time (Sec. IV's Delta t_max / Delta t_av with
     CTAs as the workers), else 0 */
  double zc_dt_max_over_avg;
  double eps_eri;           /* the ERI screen's threshold in this build (< 0: off) */
  int64_t n_eri_removed;    /* quadruples (A, B, F, G) the ERI screen removed */
} hfx_stats_v1;

hfx_status hfx_stats(const hfx_ctx *ctx, void *stats);

/*
 * One exchange term, contracted on the GPU without allocating any device
 * memory.  The paper has no counterpart to this entry point; it exists for
 * callers that cannot allocate device memory at call time -- a host framework
 * that owns the GPU's memory through its own pool and forbids direct
 * cudaMalloc, a latency-critical loop where cudaMalloc/cudaFree (which may
 * synchronize the device) are not allowed, or a process whose device memory is
 * already fully reserved by another allocator.
 *
 * Computes, on cuda_stream (NULL = legacy default stream),
 *   out[i][j] = sum_{alpha,beta,k,l} cA[alpha][i][k] V[alpha][beta] cB[beta][j][l] D[k][l]
 * in the C((VC)D) order the build uses (Y = V cB, T = Y D, out = cA T).  The
 * exchange matrix receives minus this term.
 *   cA  [nabf_a][nao_i][nao_k]   V [nabf_a][nabf_b]
 *   cB  [nabf_b][nao_j][nao_l]   D [nao_k][nao_l]    out [nao_i][nao_j]
 * All pointers are device memory on the current device, row-major FP64, owned
 * by the caller; out is overwritten.
 *
 * Working memory: the two intermediates Y and T live in one fixed 2 MiB static
 * device array (each at most 131072 doubles: nabf_a*nao_j*nao_l and
 * nabf_a*nao_j*nao_k must both be <= 131072, else HFX_E_SHAPE).  Every GPU
 * that loads the library holds that array until the process exits.  The first
 * call on each device looks the array's address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * address is kept per device and per CUDA context: after cudaDeviceReset, or
 * with another context current, the next call looks it up again, so that call
 * too must come before any stream capture.  No call allocates or frees device
 * memory.  All calls share the one array:
 * calls whose kernels overlap on the GPU (different streams, or different host
 * threads on one device) race on it and give wrong results -- order them on
 * one stream.  Each call writes every intermediate element it reads, so
 * nothing from an earlier call leaks into the result.
 *
 * The call is asynchronous: results are in out once the stream reaches them.
 * Errors: HFX_E_ARG (null pointer, size < 1), HFX_E_SHAPE (intermediates
 * larger than the static array, or nao_i*nao_j > 2^31 - 1), HFX_E_CUDA
 * (device lookup or launch failed).
 */
hfx_status hfx_term_noalloc(int32_t nabf_a, int32_t nabf_b, int32_t nao_i, int32_t nao_k,
                            int32_t nao_j, int32_t nao_l, const double *cA, const double *V,
                            const double *cB, const double *D, double *out, void *cuda_stream);

/*
 * Self-check of the split-precision tensor-core product used by HFX_OZAKI
 * (the matrix products of Appendix A's C((VC)D) chain):
 *   C[M][N] = A[M][K] B[K][N]  (host, row-major FP64), 1 <= K <= 640,
 * computed from nslices (1..6) balanced base-128 digits per operand row with
 * exact tensor-core group sums (see the header of the library's Ozaki
 * kernels).  Allocates its own temporary device memory.  Errors: HFX_E_ARG,
 * HFX_E_NOMEM, HFX_E_CUDA, HFX_E_TIMEOUT.
 */
hfx_status hfx_selftest_ozaki(int32_t M, int32_t N, int32_t K, const double *A, const double *B,
                              double *C, int32_t nslices);

/*
 * Failure-detection self-test (no counterpart in the paper): launches one
 * thread that waits on a shared-memory mbarrier that nothing ever arrives at,
 * through the same bounded wait every tensor-core kernel uses, with a limit
 * of limit_cycles SM clocks (1 .. 2e9).  The wait expires, the kernel records
 * the timeout in its error word and returns normally, and so does this call:
 * HFX_E_TIMEOUT is the expected result, with *waited_cycles (if not NULL) set
 * to the clocks the kernel spent in the wait.  The CUDA context stays usable.
 * Errors: HFX_E_ARG (limit out of range), HFX_E_CUDA.
 */
hfx_status hfx_selftest_timeout(int64_t limit_cycles, int64_t *waited_cycles);

/*
 * Diagnostic (no counterpart in the paper): the measured FP64 rates that
 * bound the HFX_FP64 mode on the current device.  Every SM runs warps that
 * issue long chains of independent FP64 multiply-adds, once as DFMA on CUDA
 * cores and once as FP64 tensor-core products (mma.sync m8n8k4 f64), each
 * timed with CUDA events after a warm-up run; writes the achieved TFLOP/s
 * (2 flops per multiply-add) of each.  Allocates a small temporary buffer.
 * Errors: HFX_E_ARG (NULL outputs), HFX_E_NOMEM, HFX_E_CUDA.
 */
hfx_status hfx_probe_fp64(double *dfma_tflops, double *dmma_tflops);

/* Message for the last failing call on ctx (never NULL; "" when none). */
const char *hfx_last_error(const hfx_ctx *ctx);

/*
 * Real-space density-matrix blocks from Kohn-Sham eigenvectors (Sec. II,
 * Eq. DM_realspace), in FP64 on the GPU.  For each requested key (K, L, n):
 *   D_{Kk,Ll}(n) = (1/nk) sum_q sum_b occ[q][b] c_q[Kk][b] conj(c_q[Ll][b])
 *                  exp(2 pi i kfrac_q . n),
 * the real part (D is real for time-reversal-symmetric inputs).
 *   nk        number of k points, >= 1
 *   kfrac     nk x 3 k points in fractional reciprocal coordinates (host)
 *   nbands    bands per k point, >= 1
 *   coef      nk x nbasis x nbands complex eigenvector coefficients as (re, im)
 *             pairs, row (Kk) = basis index sum_{x<K} nao(x) + k (host)
 *   occ       nk x nbands occupation numbers (host)
 *   nkeys, keys  nkeys x 5 block keys (K, L, n1, n2, n3), |n| <= 127 (host)
 *   out       the blocks [nao(K)][nao(L)] row-major, packed in key order (host)
 *   max_imag  (nullable) receives the largest |imaginary part| dropped
 * The result can be passed to hfx_set_many('D', ...).  Ownership: inputs are
 * read during the call.  Errors: HFX_E_ARG (sizes, keys, non-finite input),
 * HFX_E_NOMEM, HFX_E_CUDA.
 */
hfx_status hfx_density_from_eigvecs(hfx_ctx *ctx, int32_t nk, const double *kfrac,
                                    int32_t nbands, const double *coef, const double *occ,
                                    int64_t nkeys, const int32_t *keys, double *out,
                                    double *max_imag);

/*
 * The last build's exchange matrix at k points (Eq. Ham_rs2kspace), FP64 on
 * the GPU:
 *   Sigma_{Ii,Jj}(k) = sum over the Sigma keys (I, J, n) of
 *                      exp(2 pi i kfrac . n) Sigma(I, J, n)_{ij}.
 *   nk, kfrac  as in hfx_density_from_eigvecs (host)
 *   out        nk x nbasis x nbasis complex as (re, im) pairs, row-major (host)
 * Errors: HFX_E_ARG, HFX_E_STATE (no build), HFX_E_NOMEM, HFX_E_CUDA.
 */
hfx_status hfx_sigma_k(hfx_ctx *ctx, int32_t nk, const double *kfrac, double *out);

/* Free the context and all device memory it owns.  NULL is allowed. */
void hfx_destroy(hfx_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HFX_H */
