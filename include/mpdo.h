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

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpdo_ctx* mpdo_t;
typedef struct mpdo_chanset* mpdo_chan_t;
typedef struct mpdo_graph* mpdo_graph_t;

typedef enum {
  MPDO_OK = 0,
  MPDO_EINVAL = 1,   /* bad argument (size, index, non-Hermitian or non-finite chi, ...) */
  MPDO_ENOMEM = 2,   /* device or host allocation failed */
  MPDO_ENOTCP = 3,   /* process matrix is not completely positive (negative Choi mass > 1e-8) */
  MPDO_ENOTTP = 4,   /* process matrix is not trace preserving (|Tr chi - 1| > 1e-8 or sum K^H K != I) */
  MPDO_ENOCONV = 5,  /* a readout came out non-finite */
  MPDO_ETIMEOUT = 6, /* reserved */
  MPDO_ECUDA = 7,    /* CUDA runtime error */
  MPDO_ESTATE = 8    /* call not valid in the handle's current state (e.g. during capture) */
} mpdo_status;

typedef enum {
  MPDO_FP64 = 0,  /* complex128 contractions, FP64 eigensolvers */
  MPDO_MIXED = 1, /* complex64 contractions, FP64 eigensolvers for the truncations */
  MPDO_FP32 = 2   /* complex64 contractions, FP32 eigensolvers */
} mpdo_prec;

enum {
  MPDO_EXPECT_TRACE = 0,     /* Tr rho, 1 value per chain (unnormalised; truncation lowers it) */
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
/* Wait for the handle's stream. */
mpdo_status mpdo_sync(mpdo_t h);

/* chi -> Kraus (Sec. III): Lambda = sum_mn chi_mn |s_m>><<s_n|, Lambda = sum_i eta_i |psi_i><psi_i|,
 * K_i = sqrt(eta_i) unvec(psi_i), in descending eta; eta <= tol * max eta is pruned (tol <= 0 means
 * 1e-12).  chi: host, (4^nq x 4^nq) complex per channel, `count` channels back to back.  Checks:
 * Hermitian and finite (EINVAL), |Tr chi - 1| <= 1e-8 and sum K^H K = I within 1e-8 (ENOTTP),
 * negative Choi mass <= 1e-8 (ENOTCP).  n_kraus (host, nullable) receives count ranks.  The Kraus
 * sets are padded with zero operators to the largest rank of the set. */
mpdo_status channel_from_process_matrix(mpdo_t h, int nq, const double* chi, double tol, mpdo_chan_t* out,
                                        int* n_kraus);
mpdo_status channel_set_from_process_matrices(mpdo_t h, int nq, int count, const double* chi, double tol,
                                              mpdo_chan_t* out, int* n_kraus);
/* Copy channel idx's Kraus operators (padded count r_pad x d x d complex) to host `out`. */
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
/* Batched forms: U_dev = device array of batch gate matrices (complex128, row-major), chan_idx_dev =
 * device int[batch] choosing each chain's channel in ch (NULL: chain b uses channel b, or channel 0
 * for a one-channel set).  Both pointers are read when the work runs (capturable). */
mpdo_status apply_1q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev);
mpdo_status apply_2q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev);
/* Truncate qubit q's Kraus leg to kappa (<= 0: kappa_max), Eq. svdNoise.  discarded (host, nullable)
 * receives batch relative discarded weights (synchronises when non-NULL). */
mpdo_status truncate_kraus(mpdo_t h, int q, int kappa, double* discarded);
/* Readouts (Sec. II.C local densities, Eqs. maxcut / maxcut_obj); out: host, see MPDO_EXPECT_*. */
mpdo_status expect(mpdo_t h, int kind, const int* args, int nargs, double* out);

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
 * that sites left of it are left-isometric and sites right of it right-isometric. */
mpdo_status mpdo_get_site(mpdo_t h, int chain, int q, double* out, int* dims);
mpdo_status mpdo_set_site(mpdo_t h, int q, int dl, int dn, int dr, const double* data);
mpdo_status mpdo_set_centre(mpdo_t h, int q);

/* When enabled, a noisy 1q gate on a site next to the orthogonality centre truncates its Kraus leg
 * through the centre's environment (the Gram of the centre over the shared bond) instead of first
 * moving the centre there with a QR step.  The kept subspace is the same as with the move (the
 * ancilla density of the site is the same matrix), so results agree up to rounding; the site is left
 * non-isometric until the next operation absorbs it (a two-qubit gate on that pair, or a centre move,
 * which then starts by moving onto it).  Useful for a sweep order in which the gate on the far site of
 * a pair is followed by the two-qubit gate on the pair.  Off by default; capturable (the setting is
 * read when each call is made). */
mpdo_status mpdo_set_neighbour_truncation(mpdo_t h, int enable);

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
 *   7  the Kraus-leg eigensolver of every kappa truncation (top kappa of G) */
#define MPDO_PROFILE_CLASSES 8
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
 *   ranks_dev device output, count ints
 *   stream    cudaStream_t the work is enqueued on (returns without waiting)
 * Returns MPDO_EINVAL for nq not in {1, 2}, count < 1 or count > MPDO_NOALLOC_MAX_CHANNELS; inputs
 * are not validated (no host copy exists).  It calls no allocating routine.  The first call on a
 * device looks up the array's device address (once per device, with that device current); make
 * that first call before any stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (different streams, or several host threads) race; serialise them. */
#define MPDO_NOALLOC_MAX_CHANNELS 64
mpdo_status channel_kraus_noalloc(int nq, int count, const double* chi_dev, double tol, double* kraus_dev,
                                  int* ranks_dev, void* stream);

/* In the complex64 modes, products with at least 128 rows and 64 columns, an inner dimension of at
 * most 2048 and a non-Hermitian result run on the tensor cores (tcgen05.mma, each FP32 operand split
 * into two TF32 parts, three TF32 products per real product, FP32 accumulation); the others, and
 * every product when this is off, run on the CUDA cores.  Off by default: the tensor cores' FP32
 * accumulation leaves about 2e-6 relative error on a 128-long product (the CUDA-core GEMM about 1e-7),
 * which takes a full-size two-qubit update past 1e-6.  No effect in MPDO_FP64. */
mpdo_status mpdo_set_tensor_cores(mpdo_t h, int enable);

/* Diagnostic: multiplies random complex64 M x K and K x N matrices with the tensor-core GEMM (tcgen05,
 * TF32 split into hi + lo parts, FP32 accumulation) and with the CUDA-core GEMM, and returns the
 * largest entry-wise difference relative to the largest entry, and the kernel's wait-timeout flag. */
mpdo_status mpdo_tc_selftest(int M, int N, int K, double* max_rel_err, int* err_flag);

/* Number of kernels the library launched on this handle since creation (for accounting). */
long long mpdo_launch_count(mpdo_t h);
const char* mpdo_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MPDO_H */
