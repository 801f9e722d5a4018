/* C ABI of the GB300 (sm_103a) MPDO noisy-circuit library.
 *
 * The library simulates noisy quantum circuits with a matrix product density operator (MPDO):
 * one rank-4 site tensor T[l, p, n, r] per qubit (left bond, physical index, Kraus leg, right
 * bond; Sec. II.C of "Tomography-assisted noisy quantum circuit simulator using matrix product
 * density operators").  Channels are given as Pauli-basis process matrices (Eq. chi, Sec. III)
 * and converted to Kraus operators through their Choi matrix on the GPU.  Every gate is followed
 * by its channel (K_i = N_i U, Sec. II.C), adds a Kraus leg, and is truncated back to chi_max on
 * the bond (Fig. 3b) and kappa_max on the Kraus leg (Eq. svdNoise, Fig. 3a).
 *
 * Conventions
 *   - Complex arrays are interleaved (re, im) doubles, row-major.
 *   - Two-qubit matrices use the basis index 2*p_q + p_{q+1}; a two-qubit Pauli index is 4*a + b
 *     with a acting on the first qubit; Pauli order I, X, Y, Z (unnormalised, so Tr chi = 1).
 *   - A handle holds `batch` independent chains of n qubits that receive the same sequence of
 *     gate positions (the gate matrices and channels may differ per chain).
 *   - Host pointers are read before the call returns; the caller keeps ownership.  Pointers named
 *     *_dev are device pointers that must stay valid until the work on the handle's stream is done.
 *   - Calls enqueue work on the handle's CUDA stream and return without waiting, except the
 *     channel constructors and `expect`/`mpdo_sync`, which synchronise the stream.
 *   - Every call returns an mpdo_status; outputs are written only on MPDO_OK.  No exception or
 *     abort crosses the boundary.  A CUDA error is reported as MPDO_ECUDA and leaves the handle
 *     in an unspecified state (free it).
 *   - Bond and Kraus dimensions follow from the gate sequence alone (min of the cap and the
 *     structural rank of the matrix being split), so no call reads data back to decide a size.
 */
#ifndef MPDO_H
#define MPDO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpdo_ctx* mpdo_t;
typedef struct mpdo_chanset* mpdo_chan_t;
typedef struct mpdo_graph* mpdo_graph_t;
typedef struct mpdo_batch* mpdo_batch_t;

typedef enum {
  MPDO_OK = 0,
  MPDO_EINVAL = 1,   /* bad argument (size, index, non-Hermitian or non-finite chi, ...) */
  MPDO_ENOMEM = 2,   /* device or host allocation failed */
  MPDO_ENOTCP = 3,   /* process matrix is not completely positive (negative Choi mass > 1e-8) */
  MPDO_ENOTTP = 4,   /* process matrix is not trace preserving (|Tr chi - 1| > 1e-8 or sum K^H K != I) */
  MPDO_ENOCONV = 5,  /* an eigensolver (truncation or chi -> Kraus) produced non-finite or collapsed
                        eigenpairs, or a readout came out non-finite */
  MPDO_ETIMEOUT = 6, /* a bounded wait inside a kernel (tensor-core pipelines) ran out */
  MPDO_ECUDA = 7,    /* CUDA runtime error */
  MPDO_ESTATE = 8,   /* call not valid in the handle's current state (e.g. during capture) */
  MPDO_EDRIFT = 9    /* the trace guard (mpdo_set_trace_guard) saw Tr rho grow, or turn negative or
                        non-finite, over one call */
} mpdo_status;

typedef enum {
  MPDO_FP64 = 0,  /* complex128 contractions, FP64 eigensolvers */
  MPDO_MIXED = 1, /* complex64 contractions, FP64 eigensolvers for the truncations */
  MPDO_FP32 = 2   /* complex64 contractions, FP32 eigensolvers */
} mpdo_prec;

enum {
  MPDO_EXPECT_TRACE = 0,     /* Tr rho, 1 value per chain (unnormalised; truncation lowers it; the
                              * stored sites are kept near unit scale by exact powers of two per
                              * chain, which this readout multiplies back in; 0 below the FP64 range) */
  MPDO_EXPECT_ZZ = 1,        /* args = {i, j}: <Z_i Z_j>, 1 value per chain */
  MPDO_EXPECT_ZZ_MAP = 2,    /* n*n values per chain, row-major, diagonal = 1 */
  MPDO_EXPECT_GHZ = 3,       /* <GHZ| rho |GHZ>, |GHZ> = (|0..0> + |1..1>)/sqrt 2, 1 value per chain */
  MPDO_EXPECT_MAXCUT = 4,    /* args = {i0, k0, i1, k1, ...} chain positions: sum_e (1 - <Z_i Z_k>)/2 */
  MPDO_EXPECT_PURITY = 5,    /* Tr rho^2, 1 value per chain */
  MPDO_EXPECT_DISCARDED = 6, /* 3 values per chain: cumulative discarded weight of bond and Kraus-leg
                                truncations, and the smallest relative eigenvalue gap at a cut */
  MPDO_EXPECT_DIMS = 7,      /* 2n-1 values: bond dims (n-1) then Kraus dims (n) */
  MPDO_EXPECT_PROB = 8       /* args = n bits z_0 .. z_{n-1} (0 or 1): <z| rho |z>, the probability of
                                measuring the bitstring (Sec. IV's output distributions), 1 value per chain */
};
/* Every expectation except TRACE and DISCARDED is divided by Tr rho (Tr rho^2 by (Tr rho)^2). */

/* Create a handle with `batch` chains of n qubits in |0..0> (all dims 1) on `stream`
 * (a cudaStream_t, NULL = legacy default stream) of the current device.
 * chi_max >= 1 caps bonds, kappa_max >= 1 caps Kraus legs; prec is an mpdo_prec.
 * Device memory for every intermediate is allocated here (none later, except PURITY). */
mpdo_status mpdo_init(int n, int chi_max, int kappa_max, int prec, void* stream, mpdo_t* out);
mpdo_status mpdo_init_batch(int batch, int n, int chi_max, int kappa_max, int prec, void* stream, mpdo_t* out);
mpdo_status mpdo_free(mpdo_t h);
/* Back to |0..0> with zero discarded weight. Capturable. */
mpdo_status mpdo_reset(mpdo_t h);
/* Wait for the handle's stream.  Kernels record failures in a status word of the handle; this call
 * and `expect` read and clear it: MPDO_ENOCONV when an eigensolver produced non-finite or collapsed
 * eigenpairs since the last read (for example from non-finite site data), MPDO_ETIMEOUT when a
 * kernel's bounded wait ran out (the kernel skipped its output; the handle's state is unspecified). */
mpdo_status mpdo_sync(mpdo_t h);

/* chi -> Kraus (Sec. III): Lambda = sum_mn chi_mn |s_m>><<s_n|, Lambda = sum_i eta_i |psi_i><psi_i|,
 * K_i = sqrt(eta_i) unvec(psi_i), in descending eta; eta <= tol * max eta is pruned (tol <= 0 means
 * 1e-12).  nq = 1, 2 or 3 (three-qubit channels for apply_3q).  chi: host, (4^nq x 4^nq) complex per
 * channel, `count` channels back to back.  Checks:
 * Hermitian and finite (EINVAL), |Tr chi - 1| <= 1e-8 and sum K^H K = I within 1e-8 (ENOTTP),
 * negative Choi mass <= 1e-8 (ENOTCP).  n_kraus (host, nullable) receives count ranks.  The Kraus
 * sets are padded with zero operators to the largest rank of the set. */
mpdo_status channel_from_process_matrix(mpdo_t h, int nq, const double* chi, double tol, mpdo_chan_t* out,
                                        int* n_kraus);
mpdo_status channel_set_from_process_matrices(mpdo_t h, int nq, int count, const double* chi, double tol,
                                              mpdo_chan_t* out, int* n_kraus);
/* Copy channel idx's Kraus operators (r_pad x d x d complex, r_pad = the largest rank of the set) to
 * host `out`, which must hold that many. */
mpdo_status channel_kraus(mpdo_chan_t ch, int idx, double* out, int* r_pad);
mpdo_status channel_free(mpdo_chan_t ch);

/* Noisy single-qubit gate on qubit q: K_i = N_i U (U host, 2x2 complex), a new Kraus leg, then the
 * Kraus leg is truncated to kappa_max (Eq. svdNoise) with the orthogonality centre on q.  With a
 * set of `batch` channels chain b uses channel b; with one channel every chain uses it. */
mpdo_status apply_1q(mpdo_t h, int q, const double* U, mpdo_chan_t ch);
/* Noisy two-qubit gate on (q, q+1) (U host, 4x4 complex): the two sites are merged, the gate and its
 * channel applied with the new Kraus leg on site q+1, the bond split keeping chi_max singular values
 * (Fig. 3b), and site q+1's Kraus leg truncated to kappa_max.  The centre ends on q+1. */
mpdo_status apply_2q(mpdo_t h, int q, const double* U, mpdo_chan_t ch);
/* Noisy three-qubit gate on (q, q+1, q+2) (U host, 8x8 complex, qubit q most significant), for a
 * three-qubit channel such as the crosstalk channel a tomography of a two-qubit gate together with its
 * neighbour yields (Fig. 13b; up to 64 Kraus operators).  The centre is moved onto q, the three sites
 * merged, the gate and channel applied with the new Kraus leg on site q+2, the bonds (q, q+1) and
 * (q+1, q+2) split in turn keeping chi_max values each (Fig. 3b), and site q+2's Kraus leg truncated to
 * kappa_max.  The centre ends on q+2.  The first call allocates the update's workspace (about
 * 1536 chi_max^2 kappa_max^2 elements per chain; MPDO_ENOMEM if it does not fit, MPDO_ESTATE inside a
 * capture).  Its eigenproblems are of order up to 2 chi_max kappa_max and 64 kappa_max, so the handle
 * needs 2 chi_max kappa_max <= 512 and kappa_max <= 8 (MPDO_EINVAL otherwise). */
mpdo_status apply_3q(mpdo_t h, int q, const double* U, mpdo_chan_t ch);
/* Batched forms: U_dev = device array of batch gate matrices (complex128, row-major), chan_idx_dev =
 * device int[batch] choosing each chain's channel in ch (NULL: chain b uses channel b, or channel 0
 * for a one-channel set).  Both pointers are read when the work runs (capturable). */
mpdo_status apply_1q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev);
mpdo_status apply_2q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev);
mpdo_status apply_3q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev);
/* Truncate qubit q's Kraus leg to kappa (<= 0: kappa_max), Eq. svdNoise.  discarded (host, nullable)
 * receives batch relative discarded weights (synchronises when non-NULL). */
mpdo_status truncate_kraus(mpdo_t h, int q, int kappa, double* discarded);
/* Global bond truncation of Sec. II.D (Fig. 3b), the paper's own schedule: QR decompositions from
 * left to right bring the chain into canonical form, then every bond is truncated to chi (>= 1)
 * Schmidt values from right to left, each by the eigen-decomposition of its Gram matrix with the
 * centre on the bond's right site.  The centre ends on site 0.  To run this schedule, create the
 * handle with chi_max large enough that the per-gate splits keep every bond's rank, and call this
 * after each layer of gates.  discarded (host, nullable) receives batch summed relative discarded
 * weights of this sweep (synchronises when non-NULL).  MPDO_EINVAL for chi < 1. */
mpdo_status truncate_bonds(mpdo_t h, int chi, double* discarded);
/* Readouts (Sec. II.C local densities, Eqs. maxcut / maxcut_obj); out: host, see MPDO_EXPECT_*. */
mpdo_status expect(mpdo_t h, int kind, const int* args, int nargs, double* out);

/* The whole bitstring distribution <z| rho |z> / Tr rho of every chain (the output distribution the
 * paper compares with measured data, Sec. IV.A, and between truncation settings, Sec. IV.C): out (host)
 * receives batch x 2^n values, chain-major, bitstring index with qubit 0 most significant.  All 2^q
 * prefixes of a chain are carried through site q at once (4 n batched products per chain).  n <= 15
 * (MPDO_EINVAL otherwise); MPDO_ENOMEM if the prefix environments do not fit; synchronises. */
mpdo_status mpdo_distribution(mpdo_t h, double* out);
/* Jensen-Shannon divergence of two distributions over len outcomes (natural log; both normalised
 * first; 0 log 0 = 0): the distance the paper fits noise models with (Sec. IV.A).  0 for equal
 * distributions, ln 2 for disjoint supports.  Host computation, no GPU.  MPDO_EINVAL for negative or
 * non-finite entries or a zero total. */
mpdo_status mpdo_jsd(const double* p, const double* q, int len, double* out);

/* Uhlmann fidelity F(rho, sigma) = (tr sqrt(sqrt(rho) sigma sqrt(rho)))^2 (Sec. IV.C, Eq. fidelity)
 * between chain chain_a of a and chain chain_b of b, both normalised to unit trace; the paper uses it
 * to compare truncated with untruncated states.  Dense and in FP64 whatever the handles' precision:
 * each chain's 2^n x 2^n density matrix is contracted from its sites, so n <= 7 (MPDO_EINVAL
 * otherwise, or when an intermediate of the contraction would exceed 2 GB).  Synchronises both
 * handles, allocates its temporaries and frees them before returning; MPDO_ESTATE during capture. */
mpdo_status mpdo_fidelity(mpdo_t a, int chain_a, mpdo_t b, int chain_b, double* out);

/* Checkpoint: dims, centre, discarded weights and every site tensor of every chain (versioned). */
mpdo_status mpdo_save(mpdo_t h, const char* path);
mpdo_status mpdo_load(const char* path, void* stream, mpdo_t* out);

/* CUDA-graph capture of the calls made between begin and end on this handle.  With restore != 0 the
 * end call also moves the centre and the site storage back to where they were at begin, so the
 * graph can be replayed on a state with the same dims (MPDO_ESTATE if the dims differ). */
mpdo_status mpdo_capture_begin(mpdo_t h);
mpdo_status mpdo_capture_end(mpdo_t h, int restore, mpdo_graph_t* out);
mpdo_status mpdo_graph_launch(mpdo_graph_t g);
mpdo_status mpdo_graph_free(mpdo_graph_t g);

/* Site tensors.  get: chain `chain`'s site q as complex128 [l][p][n][r] into host `out` (sized
 * dl*2*dn*dr) and its dims into dims[3] = {dl, dn, dr}; synchronises.  set: overwrite site q of every
 * chain (host data = batch blocks of dl*2*dn*dr complex) with the given dims; the neighbouring bonds
 * must match (bond q must equal dl, bond q+1 must equal dr, 1 at the ends), dl, dr <= chi_max,
 * dn <= kappa_max.  set_centre declares which site is the orthogonality centre: the caller guarantees
 * that sites left of it are left-isometric and sites right of it right-isometric.  The tensors are the
 * stored ones: the represented state is their product times the chain's power-of-two scale (see
 * MPDO_EXPECT_TRACE), which normalised readouts do not see and set_site leaves as it is. */
mpdo_status mpdo_get_site(mpdo_t h, int chain, int q, double* out, int* dims);
mpdo_status mpdo_set_site(mpdo_t h, int q, int dl, int dn, int dr, const double* data);
mpdo_status mpdo_set_centre(mpdo_t h, int q);

/* Order of the two truncations of a two-qubit update (Sec. II.D leaves the schedule open):
 *   MPDO_TRUNC_SPLIT_FIRST (default): split the merged pair's bond to chi_max (Fig. 3b), then truncate
 *     site q+1's Kraus leg, r_k kappa wide, to kappa_max (Eq. svdNoise);
 *   MPDO_TRUNC_KRAUS_FIRST: truncate the merged tensor's new Kraus leg to kappa_max first (Eq. svdNoise
 *     applied to the two-site tensor), then split the bond; the split sees a kappa-wide leg, which
 *     takes about 2.4 times fewer multiply-adds at chi = 64, kappa = 8, r_k = 16.
 * The two orders keep the same state when the bond is not cut; otherwise they are different
 * approximations.  Read when each apply_2q call is made (capturable); MPDO_EINVAL for other values. */
enum { MPDO_TRUNC_SPLIT_FIRST = 0, MPDO_TRUNC_KRAUS_FIRST = 1 };
mpdo_status mpdo_set_trunc_order(mpdo_t h, int order);

/* When enabled, a noisy 1q gate on a site next to the orthogonality centre truncates its Kraus leg
 * through the centre's environment (the Gram of the centre over the shared bond) instead of first
 * moving the centre there with a QR step.  The kept subspace is the same as with the move (the
 * ancilla density of the site is the same matrix), so results agree up to rounding; the site is left
 * non-isometric until the next operation absorbs it (a two-qubit gate on that pair, or a centre move,
 * which then starts by moving onto it).  Useful for a sweep order in which the gate on the far site of
 * a pair is followed by the two-qubit gate on the pair.  Off by default; capturable (the setting is
 * read when each call is made). */
mpdo_status mpdo_set_neighbour_truncation(mpdo_t h, int enable);

/* Trace guard, a debugging aid: with tol > 0, every apply_* and truncate_* call made outside graph
 * capture reads Tr rho of every chain afterwards (the TRACE readout, so the call synchronises) and
 * compares it with the value after the previous guarded call.  The channels are trace preserving and
 * a truncation only removes weight, so Tr rho never grows in exact arithmetic: the call returns
 * MPDO_EDRIFT (after its work is done) when a chain's trace exceeds the previous one by more than
 * tol relative, or is negative or non-finite.  Rounding moves the trace by about 1e-6 relative per
 * call in the complex64 modes and 1e-12 in FP64, and an accepted channel may be trace preserving to
 * 1e-8 only: 1e-4 and 1e-7 are suitable tolerances.  Enabling takes the current traces as the
 * baseline, mpdo_reset sets it to 1; an edit of the state between guarded calls (mpdo_set_site) is
 * measured at the next guarded call, so call this again after such an edit to take a new baseline.
 * tol <= 0 switches the guard off (the default).  MPDO_ESTATE during capture. */
mpdo_status mpdo_set_trace_guard(mpdo_t h, double tol);

/* Device memory the PURITY readout may hold for its intermediates, in bytes (0, the default: 35% of
 * the device memory free at its first call).  The purity contraction carries a chi^4 environment
 * and intermediates of up to 2 kappa chi^5 elements per site; they are processed in chunks of one
 * environment index sized to this budget, so a smaller budget means more, smaller launches and
 * the same result.  The buffers are kept until the handle is freed or the budget changes.
 * MPDO_ENOMEM if not even one chunk fits; MPDO_ESTATE during capture. */
mpdo_status mpdo_set_purity_memory(mpdo_t h, long long bytes);

/* Per-launch CUDA-event timing by kernel class, for measurement: enable records an event pair
 * around every launch made outside graph capture; read synchronises and returns, per class, the
 * summed milliseconds, the summed algorithmic flops the engine attributes to those launches (8 real
 * flops per complex multiply-add) and the launch count (arrays of MPDO_PROFILE_CLASSES), then clears
 * the record.  Classes 0-3 partition every launch (GEMM, QR, eigensolver, other); classes 4-7 are
 * subsets of them, one call site each:
 *   4  the Kraus-leg Gram G = conj(X) X^T of every kappa truncation (GEMM)
 *   5  the product X = Y A2 of a two-qubit update, the gate and channel applied to the right site (GEMM)
 *   6  the bond eigensolver of a two-qubit update (top chi of F')
 *   7  the Kraus-leg eigensolver of every kappa truncation (top kappa of G)
 *   8  the two site-streaming products of every one-qubit update (the site's bond Gram and the
 *      product with the folded gate); HBM-bound, so its second array entry holds the algorithmic
 *      bytes (the site read twice, the new site written once) instead of flops */
#define MPDO_PROFILE_CLASSES 9
mpdo_status mpdo_profile(mpdo_t h, int enable);
mpdo_status mpdo_profile_read(mpdo_t h, double* ms, double* flops, long long* count);

/* Allocation-free chi -> Kraus conversion, for callers that cannot call cudaMalloc (a plug-in
 * living inside another application's memory pool, or code that must not grow its device footprint
 * after start-up).  The paper has no counterpart: it is the same conversion as
 * channel_set_from_process_matrices, with every intermediate kept in one fixed device array
 * compiled into the library (MPDO_NOALLOC_MAX_CHANNELS channels, about 1.6 MB, held on every GPU
 * that loads the library until the process exits) instead of fresh allocations.
 *   chi_dev   device, count x (4^nq x 4^nq) complex, row-major (same layout as the host variant)
 *   kraus_dev device output, count x 4^nq Kraus operators of 2^nq x 2^nq complex (descending weight,
 *             pruned ones zeroed: eta <= tol * max eta, tol <= 0 means 1e-12)
 *   ranks_dev device output, count ints: the Kraus rank, or -1 when the process matrix is not
 *             completely positive (negative Choi mass > 1e-8) and -2 when the converted set is not
 *             trace preserving (|sum K^H K - I| > 1e-8); that channel's operators are then zero
 *   stream    cudaStream_t the work is enqueued on (returns without waiting)
 * Returns MPDO_EINVAL for nq not in {1, 2}, count < 1 or count > MPDO_NOALLOC_MAX_CHANNELS; the
 * inputs are checked on the device only (the sentinel ranks above; no host copy exists).  It calls
 * no allocating routine.  The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (different streams, or several host threads) race; serialise them. */
#define MPDO_NOALLOC_MAX_CHANNELS 64
mpdo_status channel_kraus_noalloc(int nq, int count, const double* chi_dev, double tol, double* kraus_dev,
                                  int* ranks_dev, void* stream);

/* In the complex64 modes (MIXED, FP32) the dense complex products with at least 128 rows, 64 columns
 * and an inner dimension of 16 run on the tensor cores (tcgen05.mma kind::tf32): each FP32 operand is
 * split into TF32 hi and lo parts (three real products per real product, four real products per
 * complex product), and the tensor-memory accumulator is folded every 16 k into compensated FP32
 * sums, so the error matches the CUDA-core GEMM's.  On by default in those modes (the handle holds
 * workspaces for the split operands, sized at creation); 0 keeps every product on the CUDA cores.
 * No effect in MPDO_FP64.  MPDO_ESTATE during capture when it would allocate. */
mpdo_status mpdo_set_tensor_cores(mpdo_t h, int enable);

/* Diagnostic: multiplies random complex64 M x K and K x N matrices (M >= 128, N >= 64, K >= 16) with
 * the tensor-core GEMM and with the CUDA-core GEMM, and returns the largest entry-wise difference
 * relative to the largest entry, and the tensor-core kernel's status word (2 = a wait timed out). */
mpdo_status mpdo_tc_selftest(int M, int N, int K, double* max_rel_err, int* err_flag);

/* Diagnostic: one thread waits on a shared-memory mbarrier that nothing arrives on, with the same
 * time-bounded wait the tensor-core kernels use, limited to limit_us microseconds (1 .. 1e6).  The
 * wait gives up, the kernel records the timeout in a status word and returns: MPDO_ETIMEOUT, with
 * the word in *status_out.  Demonstrates that no wait in the library can hang the GPU. */
mpdo_status mpdo_wait_selftest(int limit_us, int* status_out);

/* ---- Address-checked debug build.  libmpdo_bounds.so is this library compiled from the same
 * sources with -DMPDO_BOUNDS (paper_2508_07610_gb300.build.build(bounds=True)).  In it every global
 * memory access of the MPDO kernels first checks that its bytes lie inside a live device range: an
 * allocation the library made, or a range the caller registered.  A failed check is counted, the
 * first one is recorded, and the access goes to a scratch buffer instead: no trap, no fault, and the
 * results of that call are meaningless.  The release library compiles none of this.
 *
 * mpdo_bounds_enabled: 1 in the checked build, 0 in the release library.
 * mpdo_bounds_register(p, bytes): a caller-owned device buffer the kernels may read (the U_dev and
 *   chan_idx_dev arrays of the batched forms, the buffers of channel_kraus_noalloc); ranges may
 *   overlap.  mpdo_bounds_unregister(p) removes the range registered at p (MPDO_EINVAL if none).
 *   Both are no-ops returning MPDO_OK in the release library.
 * mpdo_bounds_read: synchronises the device, returns the number of failed checks since the last call
 *   in *failures and clears it; the first failure's source file name (at most file_cap - 1
 *   characters), line, address and access size go to the other outputs (each nullable).  MPDO_ENOMEM
 *   when more than 16384 disjoint ranges were live at once (checking then switched off), MPDO_ESTATE
 *   in the release library. */
int mpdo_bounds_enabled(void);
mpdo_status mpdo_bounds_register(const void* p, size_t bytes);
mpdo_status mpdo_bounds_unregister(const void* p);
mpdo_status mpdo_bounds_read(unsigned long long* failures, char* file, int file_cap, int* line,
                             unsigned long long* addr, unsigned long long* bytes);

/* ---- Batched runtime: many independent noisy circuits ("instances") on one GPU.  The paper runs one
 * circuit at a time; this is the throughput form of the same per-gate update (Sec. II.C-II.D).
 * Instance c has n_qubits[c] qubits (starting in |0..0>) and the ops op_begin[c] .. op_begin[c+1]-1:
 *   op_kind[o]  1 or 2 (the gate acts on op_q[o], or on op_q[o] and op_q[o]+1; three-qubit gates
 *               are not taken by the batched runtime: use apply_3q_batch on a handle), or
 *               MPDO_OP_TRUNCATE_BONDS: the global bond truncation truncate_bonds(h, op_q[o], NULL)
 *               (1 <= op_q[o] <= chi_max; op_U and op_chi of the op are not read)
 *   op_U[o]     32 doubles: the 2x2 or 4x4 gate, complex row-major (interleaved re, im), 2x2 in the
 *               first 8 doubles
 *   op_chi[o]   index of the channel that follows the gate in the process-matrix table chis: n_chi
 *               matrices back to back, matrix m is 4^chi_nq[m] x 4^chi_nq[m] complex (Eq. chi), with
 *               chi_nq[m] equal to the op's kind
 * Instances whose gates sit on the same positions in the same order form a group; a group runs as one
 * or more handles of batched chains, each captured into one CUDA graph on its own stream.  With a
 * tuning file (nullable path), groups of at least 128 instances not yet in the file are timed over
 * every schedule (1, 2 or 4 handles; tensor cores on or off in the complex64 modes) and the fastest
 * is stored in the file as JSON; entries found in the file are used without timing.  All host arrays
 * are copied.  MPDO_EINVAL for inconsistent arrays; the channel checks of
 * channel_set_from_process_matrices apply (MPDO_ENOTCP, MPDO_ENOTTP). */
enum { MPDO_OP_TRUNCATE_BONDS = 8 };
mpdo_status mpdo_batch_create(int count, const int* n_qubits, const int* op_begin, const int* op_kind, const int* op_q,
                              const double* op_U, const int* op_chi, int n_chi, const int* chi_nq, const double* chis,
                              int chi_max, int kappa_max, int prec, const char* tuning_path, mpdo_batch_t* out);
/* Replay every instance's circuit from |0..0> (asynchronous; the groups run concurrently). */
mpdo_status mpdo_batch_run(mpdo_batch_t b);
/* Wait for the run; the first status word error of any handle (see mpdo_sync) is returned. */
mpdo_status mpdo_batch_sync(mpdo_batch_t b);
/* Per-instance readouts, out in instance order: MPDO_EXPECT_TRACE, _GHZ, _PURITY (1 value each),
 * _DISCARDED (3 each), _ZZ_MAP (n_qubits[c]^2 each, packed), _MAXCUT (1 each: instance c's edges are
 * the pairs of chain positions args[arg_begin[c]] .. args[arg_begin[c+1]-1]).  Synchronises. */
mpdo_status mpdo_batch_expect(mpdo_batch_t b, int kind, const int* arg_begin, const int* args, double* out);
/* Number of groups and handles, and the two-qubit updates of one run. */
mpdo_status mpdo_batch_info(mpdo_batch_t b, int* groups, int* handles, long long* updates_2q);
/* Schedule of group g: its qubit count, instances, handles, tensor-core setting and the tuner's time
 * per replay in ms (0 when not timed). */
mpdo_status mpdo_batch_schedule(mpdo_batch_t b, int group, int* n_qubits, int* chains, int* handles,
                                int* tensor_cores, double* tuned_ms);
/* Uhlmann fidelity (mpdo_fidelity) of every instance of a against the same instance of b, for two
 * batches built from the same circuits (typically different caps): count values in instance order.
 * Call after both have run. */
mpdo_status mpdo_batch_fidelity(mpdo_batch_t a, mpdo_batch_t b, double* out);
mpdo_status mpdo_batch_free(mpdo_batch_t b);

/* Number of kernels the library launched on this handle since creation (for accounting). */
long long mpdo_launch_count(mpdo_t h);
const char* mpdo_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MPDO_H */
