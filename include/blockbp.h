/*
 * blockbp.h -- C ABI of the GB300 blockBP decoder for the planar surface code.
 *
 * The library decodes batches of syndromes of the distance-d planar surface
 * code under i.i.d. depolarizing noise with the blockBP decoder of Kaufmann
 * and Arad, "Blockbp decoder for the surface code" (arXiv:2402.04834):
 * for each syndrome and each of the four logical cosets I, X, Y, Z it runs
 * block belief propagation with boundary-MPS messages on the coset tensor
 * network (Sec. III.D, Algorithm 1), reads the coset log-probability out with
 * the Bethe formula of Lemma 1, and picks a coset (Algorithm 1, Remark 6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice (Sec. II.B, Fig. 1): the code lives on a (2d-1) x (2d-1) grid;
 *    (even, even) = horizontal-edge qubit, (odd, odd) = vertical-edge qubit,
 *    (even, odd) = site check A_u (Z type), (odd, even) = plaquette check
 *    B_p (X type).  n = d^2 + (d-1)^2 qubits, m = 2d(d-1) checks.
 *  - Qubit order: row-major over the grid positions with i + j even.
 *  - Syndrome order: all A_(r,c) row-major (r < d, c < d-1), then all
 *    B_(r,j) row-major (r < d-1, j < d); one byte per bit, values 0/1.
 *  - Coset order: 0 = I, 1 = X, 2 = Y, 3 = Z, relative to the library's pure
 *    error f_s (X strings from a flagged A_(r,c) to the right boundary along
 *    row r, Z strings from a flagged B_(r,j) to the bottom boundary along
 *    column j).  X-bar is X on the horizontal edges of row 0, Z-bar is Z on
 *    the horizontal edges of column 0.  A decision c means the correction
 *    f_s * L_c.
 *  - Every pointer argument is owned by the caller.  "Device" pointers are
 *    CUDA global memory of the current device; "host" pointers are ordinary
 *    (preferably pinned) host memory.  Calls are asynchronous on ``stream``
 *    (a cudaStream_t, NULL = legacy default stream) unless stated otherwise.
 *  - Return value: BBP_OK (0) or a negative BBP_E* code; bbp_strerror() gives
 *    its text.  Numerical trouble of a single syndrome never fails a call:
 *    it is reported in that syndrome's flags.
 */
#ifndef BLOCKBP_H
#define BLOCKBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define BBP_OK 0
#define BBP_EINVAL (-1)        /* bad argument (null pointer, size, parameter) */
#define BBP_ECUDA (-2)         /* a CUDA runtime call failed */
#define BBP_ENOSPACE (-3)      /* workspace smaller than bbp_workspace_bytes() */
#define BBP_EUNSUPPORTED (-4)  /* (k, D, precision) outside the compiled kernels */
#define BBP_ETOOLARGE (-5)     /* batch needs more than the static workspace holds */

/* Size of the static workspace used by bbp_decode_batch_static (32 MiB). */
#define BBP_STATIC_WORKSPACE_BYTES (32u << 20)

/* Per-coset flags (bit mask, Algorithm 1 and Remark 6). */
#define BBP_FLAG_UNTRUSTED 1   /* Delta >= delta1: the Bethe value is not trusted */
#define BBP_FLAG_OVERLAP 2     /* some edge overlap <m_uv|m_vu> <= 0 */
#define BBP_FLAG_BLOCK 4       /* some block contraction Z_v <= 0 */
#define BBP_FLAG_NONFINITE 8   /* a norm or a log went non-finite */
/* An MPS bond outgrew its slot, or a register-form-only kernel met a block
 * without a register form (neither is expected; the coset's values are not
 * meaningful). */
#define BBP_FLAG_CAPACITY (1 << 16)
/* An index or size checked on the device was out of range and the access was
 * skipped (the coset's values are not meaningful): a syndrome of a mixed
 * batch whose distance lies outside 2..d_max (always checked), or, in the
 * library built with device bounds checks (-DBLOCKBP_CHECKS, whose
 * bbp_version() says so), any table index the kernels derive. */
#define BBP_FLAG_CHECK (1 << 17)

/* Algorithms. */
#define BBP_ALG_MPS 0          /* blockBP with boundary-MPS messages of bond D (Sec. III.D) */
#define BBP_ALG_FUSED 1        /* fused-block BP with dense messages of 2^k (Remark 9), k <= 6 */

/* Precisions. */
#define BBP_FP64 0             /* all arithmetic in double */
#define BBP_FP32 1             /* tensors and linear algebra in float; logs, Delta and
                                  the read-out sums in double */

/*
 * Decoder parameters (Sec. III.E "Decoder Parameters"; values of Sec. IV).
 *   d         code distance, d >= 2
 *   k         block side in tensor-network nodes (Algorithm 1 "Partition into
 *             k x k blocks"); blocks on the far edges take the remainder (Remark 1)
 *   D         maximal MPS bond dimension chi of messages and in-block contraction
 *   max_iter  maximal number of BP iterations (one iteration = two half-rounds,
 *             Remark 8)
 *   p         depolarizing probability, 0 < p < 0.75 (Sec. IV)
 *   eta       damping parameter (Remark 7; the paper uses 0.1)
 *   delta0    exit threshold on Delta (Remark 4); 0 runs exactly max_iter
 *   delta1    trust threshold on Delta (Remark 6)
 *   cutoff    relative singular-value cutoff: at every truncation the
 *             singular values below cutoff * sigma_1 are dropped as numerical
 *             zeros (the paper is silent; 1e-13 for BBP_FP64, 1e-7 for BBP_FP32)
 *   precision BBP_FP64 or BBP_FP32
 *   launch_warps, launch_cosets, launch_ctas_per_sm, launch_messages
 *             launch shape of the fused path (tuning only; results do not
 *             depend on them): warps per CTA, cosets decoded together by one
 *             CTA (1, 2 or 4; they share the block geometry and, off row 0
 *             and column 0, the node tensors), resident CTAs per SM of
 *             bbp_decode_mixed, and where the messages live (1 shared memory,
 *             2 a workspace slot per resident CTA with a persistent grid,
 *             3 shared memory with every block update in register form:
 *             k = 4 at odd d only, where every block is 4 x 4 or one node
 *             wide; small per-warp buffers, sized for more CTAs per SM; for
 *             bbp_decode_mixed only on request, see there).
 *             0 picks the first compiled shape, in order of measured speed,
 *             whose shared memory allows the CTAs per SM its registers are
 *             sized for, else the first that fits; compiled (warps, cosets):
 *             FP32 (8,4) (8,2) (4,2) (4,4) (16,1) (8,1) (4,1), of which (8,4)
 *             and (8,2) also with workspace messages and in register-form-only
 *             variants ((8,4) sized for 4 and for 3 CTAs per SM, the first
 *             whose shared memory allows it taken; (8,2) for 4); FP64 (4,2)
 *             (8,2) (8,1) (4,4), (4,2) also with workspace messages, (4,2) and
 *             (8,2) in register-form-only variants (4 and 2 CTAs per SM); for
 *             k = 5, 6
 *             (workspace messages only): FP32 (6,1) (4,1) (2,1), FP64 (3,1)
 *             (2,1); other requests give BBP_EUNSUPPORTED.
 *   algorithm BBP_ALG_MPS, or BBP_ALG_FUSED: every k x k block fused into one
 *             vertex with dense messages (Remark 9; the form the paper ran for
 *             k = 1, 2, 4).  Nothing is truncated, D and cutoff are unused,
 *             and the result equals BBP_ALG_MPS whenever that truncates
 *             nothing.  Needs k <= 6; a workspace when the messages live in
 *             workspace slots (always for k = 5, 6).
 */
typedef struct bbp_params {
  int32_t d;
  int32_t k;
  int32_t D;
  int32_t max_iter;
  double p;
  double eta;
  double delta0;
  double delta1;
  double cutoff;
  int32_t precision;
  int32_t algorithm;
  int32_t launch_warps;        /* fused path: warps per CTA (2, 3, 4, 6, 8, 16), 0 = default */
  int32_t launch_ctas_per_sm;  /* bbp_decode_mixed: resident CTAs per SM, 0 = the occupancy limit */
  int32_t launch_cosets;       /* fused path: cosets per CTA (1, 2, 4), 0 = default */
  int32_t launch_messages;     /* fused path: 1 shared memory, 2 workspace slots, 3 register form only, 0 = default */
} bbp_params;

/*
 * bbp_workspace_bytes -- device scratch needed by bbp_decode_batch for B
 * syndromes: the MPS messages of every syndrome x coset (Sec. III.D); for
 * BBP_ALG_FUSED none when the launch shape keeps the messages in shared
 * memory, else the dense messages of the resident CTAs, min(4B / G, 512)
 * slots of G x M x V scalars (G cosets per CTA, M directed block edges,
 * V = 16 for k <= 4 and 64 for k = 5, 6; d = 31, k = 6: 440 x 64 x 4 bytes
 * = 112.6 KB a slot in FP32).  With
 * include_io != 0 it also counts room for device copies of the inputs and
 * outputs, as bbp_decode_batch_host needs.  Writes the size to *bytes.
 * Errors: BBP_EINVAL for invalid parameters or a null pointer.
 */
int bbp_workspace_bytes(const bbp_params* prm, int64_t B, int include_io, size_t* bytes);

/*
 * bbp_decode_batch -- blockBP decoding of B syndromes (Algorithm 1).
 *   syndromes  device, [B][m] bytes 0/1 (order above)
 *   logp       device, [B][4] doubles: natural log of the Bethe estimate of
 *              pi(f_s L G) (Lemma 1) for the cosets I, X, Y, Z
 *   delta      device, [B][4] doubles: final Delta of each coset (Remark 4)
 *   iters      device, [B][4] int32: BP iterations run
 *   flags      device, [B][4] int32: BBP_FLAG_* bits
 *   decision   device, [B] int8: chosen coset index (Algorithm 1 / Remark 6):
 *              largest logp among unflagged cosets, else smallest Delta,
 *              ties to the lowest index
 *   workspace  device scratch of at least bbp_workspace_bytes(prm, B, 0)
 *              bytes, 256-byte aligned; contents on entry are ignored
 * Asynchronous on ``stream``.  Returns BBP_EINVAL for bad arguments,
 * BBP_ENOSPACE for a short workspace, BBP_EUNSUPPORTED when no compiled
 * kernel covers (k, D, precision), BBP_ECUDA when a launch fails.
 */
int bbp_decode_batch(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                     double* logp, double* delta, int32_t* iters, int32_t* flags,
                     int8_t* decision, void* workspace, size_t workspace_bytes,
                     void* stream);

/*
 * bbp_decode_batch_host -- the same decode with HOST buffers: copies the
 * syndromes to the device, decodes, copies every output back and
 * synchronises ``stream`` before returning.  ``workspace`` is device memory
 * of at least bbp_workspace_bytes(prm, B, 1) bytes.  Any output pointer
 * except decision may be NULL to skip its copy.  Errors as bbp_decode_batch.
 */
int bbp_decode_batch_host(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                          double* logp, double* delta, int32_t* iters, int32_t* flags,
                          int8_t* decision, void* workspace, size_t workspace_bytes,
                          void* stream);

/*
 * bbp_sample -- seeded depolarizing errors and their syndromes on the device
 * (Sec. IV workload).  Shot t in [first_shot, first_shot + B) draws, for each
 * qubit q, r = mix(mix(mix(seed) ^ t) ^ q) with mix the SplitMix64 output
 * function; identity iff (r >> 11) < floor((1 - p) 2^53), otherwise
 * ((mix(r) >> 32) * 3) >> 32 selects X, Y, Z.
 *   ex, ez      device [B][n] bytes: X and Z bit planes of the error
 *   syndromes   device [B][m] bytes
 *   true_class  device [B] int8: coset index of the error relative to f_s
 * Any of ex / ez may be NULL.  Asynchronous on ``stream``.
 */
int bbp_sample(uint64_t seed, int64_t first_shot, int64_t B, int32_t d, double p,
               uint8_t* ex, uint8_t* ez, uint8_t* syndromes, int8_t* true_class,
               void* stream);

/*
 * bbp_pure_error -- the pure error f_s of each syndrome (Algorithm 1, first
 * step, which asks for any Pauli with syndrome s; this construction is the
 * library's choice): for every flagged site check A_(r,c) an X string
 * on the horizontal edges of row r right of it, for every flagged plaquette
 * B_(r,j) a Z string on the horizontal edges of column j below it.  f_s
 * vanishes on the supports of both logicals; s(f_s) = s.
 *   d           distance, 2 <= d <= 64
 *   syndromes   device [B][m] bytes 0/1 (order above)
 *   fx, fz      device [B][n] bytes, caller-owned: X and Z bit planes, qubits
 *               in the order of bbp_sample (grid row-major over i + j even)
 * Asynchronous on ``stream``.  Errors: BBP_EINVAL for a bad d or B or a null
 * pointer (B = 0 is a no-op), BBP_ECUDA.
 */
int bbp_pure_error(int32_t d, const uint8_t* syndromes, int64_t B, uint8_t* fx, uint8_t* fz, void* stream);

/*
 * bbp_decode_batch_static -- the decode of bbp_decode_batch without any
 * allocation, for callers that cannot allocate device memory: real-time
 * loops that must not take the allocator's locks or fail for lack of memory
 * mid-run, and hosts that own only the input and output buffers.  The paper has no counterpart; this
 * is an interface of this library.
 *   Arguments and outputs are those of bbp_decode_batch, minus the workspace:
 *   the message arena is a file-scope device array of
 *   BBP_STATIC_WORKSPACE_BYTES (32 MiB) that every GPU loading the library
 *   reserves until the process exits.
 *   Size limit: the batch may need at most BBP_STATIC_WORKSPACE_BYTES of
 *   workspace (bbp_workspace_bytes(prm, B, 0)); beyond that the call returns
 *   BBP_ETOOLARGE and launches nothing (d = 11, k = 4, D = 8: up to 512
 *   syndromes in FP32, 256 in FP64).
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture begins.  With CUDA's lazy module loading (the default)
 *   that first look-up is also when the device reserves the 32 MiB, so it
 *   can fail with BBP_ECUDA when the device is out of memory: make it at
 *   start-up.  The address is cached per device ordinal for the life of the
 *   process; resetting the device (cudaDeviceReset) after a call leaves the
 *   cache stale and is not supported.  No call allocates or frees memory.
 *   Every call shares the one array, and the kernel initialises each message
 *   before it reads it, so nothing must start at zero and the last call's
 *   contents are simply overwritten.  Calls whose kernels overlap on the GPU
 *   (different streams, or several host threads) race on the array and give
 *   undefined results: serialise them.
 * Errors as bbp_decode_batch, plus BBP_ETOOLARGE.
 */
int bbp_decode_batch_static(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                            double* logp, double* delta, int32_t* iters, int32_t* flags,
                            int8_t* decision, void* stream);

/*
 * Learned warm start (fused path only).  The paper starts BP from uniform
 * messages (Remark 2); these calls let a small network propose the initial
 * message of every directed block edge instead, and train that network on
 * converged messages.  Rows are ordered (syndrome, coset, message); M is the
 * number of directed block edges (bbp_message_count).  Cold start remains
 * the default and the fallback.
 */
#define BBP_WARM_FEATURES 256        /* features per message */
#define BBP_WARM_HIDDEN 256          /* width of the two hidden layers */
#define BBP_WARM_OUT 16              /* outputs: logits of a 2^k <= 16 message */
#define BBP_WARM_MAX_ROWS 4194240    /* rows per infer / train call */
#define BBP_WARM_STATUS_OFFSET 270336 /* bbp_warm_infer: int32 status word in the workspace */
#define BBP_WARM_INFER_WORKSPACE_BYTES 270592 /* bbp_warm_infer needs this much, for any N */

/* Number of directed block edges M of (d, k). */
int bbp_message_count(const bbp_params* prm, int32_t* M);

/*
 * bbp_message_features -- features of every message of B syndromes: a 7 x 7
 * window of the coset network around the message's side, read in the frame
 * rotated so the message points right (channels: inside the grid, qubit,
 * coset-frame x bit, z bit, syndrome bit of a check), one-hot direction,
 * one-hot message length, 10 p, 1.
 *   feats  device [B*4*M][BBP_WARM_FEATURES] float
 *   lens   device [B*4*M] int32 message lengths 2^w, or NULL
 * Requires k <= 4.  Asynchronous on ``stream``.
 */
int bbp_message_features(const uint8_t* syndromes, int64_t B, const bbp_params* prm, float* feats,
                         int32_t* lens, void* stream);

/*
 * bbp_message_classes -- which feature rows of a syndrome are distinct.  The
 * four coset frames differ only on the horizontal edges of grid row 0 (the
 * X-bar string, flipped in cosets X and Y) and of grid column 0 (Z-bar,
 * flipped in Y and Z), so cosets that agree on the strings a message's 7 x 7
 * window sees have the same features, hence the same proposal: one row for
 * a window that sees neither, two for one string, four for both.  Host
 * only, no CUDA call.
 *   uniq_of  host [4][M] int32: distinct row of (coset, message)
 *   row_key  host [4*M] int32 (capacity): row u stands for (coset, message)
 *            = (row_key[u] / M, row_key[u] % M), the coset being the first
 *            of the cosets it stands for (order I, X, Y, Z)
 *   n_rows   the number U of distinct rows (d = 11, k = 4: 154 of 480)
 * Requires k <= 4.  Errors: BBP_EINVAL.
 */
int bbp_message_classes(const bbp_params* prm, int32_t* uniq_of, int32_t* row_key, int32_t* n_rows);

/*
 * bbp_message_features_rows -- bbp_message_features for the U listed rows of
 * every syndrome only: feats [B*U][BBP_WARM_FEATURES] (row b*U + u is
 * (coset, message) = row_key[u] of syndrome b, bit for bit the row that
 * bbp_message_features writes for it), lens [B*U] or NULL.  row_key is
 * device memory (from bbp_message_classes).  Asynchronous on ``stream``.
 */
int bbp_message_features_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const int32_t* row_key,
                              int32_t U, float* feats, int32_t* lens, void* stream);

/*
 * bbp_message_feature_bits_rows -- the same rows as bits: bits
 * [B*U][BBP_WARM_FEATURES / 32] uint32, bit q % 32 of word q / 32 set where
 * feature q is not zero.  Every feature is 0 or 1 except feature 253 (10 p,
 * whose bit is set), so the bits and p give the rows back exactly
 * (bbp_warm_infer_bits); 32 bytes a row instead of 1 KB.
 */
int bbp_message_feature_bits_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                                  const int32_t* row_key, int32_t U, uint32_t* bits, int32_t* lens, void* stream);

/*
 * bbp_expand_rows -- messages [B][4][M][16] from distinct rows [B*U][16]:
 * msgs[b][c][i] = rows[b*U + uniq_of[c*M + i]] (uniq_of device, from
 * bbp_message_classes).  Asynchronous on ``stream``.
 */
int bbp_expand_rows(const float* rows, int64_t B, int32_t U, const int32_t* uniq_of, int32_t M, float* msgs,
                    void* stream);

/* Parameters of the network: W1 (F x H), b1, W2 (H x H), b2, W3 (H x O), b3, row-major. */
int bbp_warm_param_count(void);

/* Device scratch of one infer or train call over N rows. */
int bbp_warm_workspace_bytes(int64_t N, size_t* bytes);

/*
 * bbp_warm_infer -- initial messages from the network: the proposal u (exp
 * of the logits over the first lens[row] entries, unit norm) is blended with
 * the uniform start, msgs = normalise((1 - alpha) uniform + alpha u), zero
 * beyond lens[row]; alpha in [0, 1] (0 = cold start).  The layers run on
 * the tensor cores (tcgen05): operands (features, weights, hidden
 * activations) rounded to BF16, FP32 accumulation.  All pointers device
 * memory; N <= BBP_WARM_MAX_ROWS; workspace 256-byte aligned.  A
 * device-side wait that gives up (none is expected) leaves NaN rows, which
 * the decoder replaces by the uniform start, and sets the int32 at byte
 * BBP_WARM_STATUS_OFFSET of the workspace to 1 (0 otherwise); the call is
 * asynchronous, so read it after the stream has finished.
 */
int bbp_warm_infer(const float* theta, const float* feats, const int32_t* lens, int64_t N, float alpha,
                   float* msgs, void* workspace, size_t workspace_bytes, void* stream);

/*
 * bbp_warm_infer_bits -- bbp_warm_infer from feature bits (as
 * bbp_message_feature_bits_rows writes them) and the noise rate p of
 * feature 253: the same BF16 operands, so the same messages bit for bit as
 * bbp_warm_infer on the FP32 rows.  Arguments and errors otherwise as
 * bbp_warm_infer (p in (0, 0.75)).
 */
int bbp_warm_infer_bits(const float* theta, const uint32_t* bits, const int32_t* lens, int64_t N, double p,
                        float alpha, float* msgs, void* workspace, size_t workspace_bytes, void* stream);

/*
 * bbp_warm_infer_syndromes -- bbp_warm_infer for every message of B
 * syndromes (device [B][m] bytes), with the features of
 * bbp_message_features computed inside the kernel instead of read from a
 * features buffer: msgs [B*4*M][16], rows ordered (syndrome, coset,
 * message), equal bit for bit to bbp_message_features followed by
 * bbp_warm_infer.  Uses prm's d, k (<= 4) and p.  Workspace and status word
 * as bbp_warm_infer; BBP_EUNSUPPORTED if the geometry's tables do not fit
 * in shared memory next to the operand tiles.  It needs no features buffer
 * (1 KB per message) and takes about 1.1x the time of the two calls (d = 11:
 * the features are computed by the 8 warps of the one CTA per SM that the
 * operand tiles allow, between the tensor-core phases).
 */
int bbp_warm_infer_syndromes(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                             float alpha, float* msgs, void* workspace, size_t workspace_bytes, void* stream);

/*
 * bbp_warm_train_step -- one FP32 training step on N rows: forward, the loss
 * 1 - <u, t>^2 per message (the Delta term of Remark 4) averaged over rows,
 * backward into grad (bbp_warm_param_count floats), and, when step > 0 and
 * adam_m / adam_v are given, one Adam update of theta with learning rate lr.
 * loss_sum receives the sum of the per-row losses.  targets [N][16] are unit
 * vectors.  All pointers device memory.
 */
int bbp_warm_train_step(float* theta, float* adam_m, float* adam_v, int32_t step, float lr, const float* feats,
                        const float* targets, const int32_t* lens, int64_t N, float* grad, float* loss_sum,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * bbp_decode_batch_ex -- bbp_decode_batch for algorithm BBP_ALG_FUSED with
 * optional initial messages init_msgs [B][4][M][16] (renormalised; an
 * all-zero message falls back to uniform) and optional export of the
 * messages after the BP loop into final_msgs [B][4][M][16] (float).
 * Errors as bbp_decode_batch; BBP_EINVAL for the MPS algorithm, and for
 * k > 4 when messages are given or asked for.  workspace: at least
 * bbp_workspace_bytes(prm, B, 0) bytes (none for k <= 4).
 */
int bbp_decode_batch_ex(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const float* init_msgs,
                        float* final_msgs, double* logp, double* delta, int32_t* iters, int32_t* flags,
                        int8_t* decision, void* workspace, size_t workspace_bytes, void* stream);

/*
 * bbp_decode_warm -- the learned decoder in one call (fused path, k <= 4):
 * features of the distinct message rows (bbp_message_classes; the features
 * of bbp_message_features_rows, held as bits: every feature is 0 or 1 but
 * 10 p), the network on the tensor cores (bbp_warm_infer, alpha as there;
 * the same BF16 operands, bit for bit), the expansion of each proposal to the
 * cosets it stands for (bbp_expand_rows), then bbp_decode_batch_ex started
 * from the proposals.  Outputs as bbp_decode_batch.
 *   theta      device, bbp_warm_param_count() floats (trained parameters)
 *   syndromes  device, [B][m] bytes 0/1
 *   workspace  device, at least bbp_decode_warm_workspace_bytes(prm, B, 0)
 *              bytes, 256-byte aligned: the network's scratch (its status
 *              word at byte BBP_WARM_STATUS_OFFSET, as for bbp_warm_infer),
 *              the class tables, the features of the distinct rows (32
 *              bytes per row; d = 11, k = 4: 154 rows per syndrome), the
 *              proposals, the expanded initial messages (B x 4 x M x 16
 *              floats) and the decode's own workspace
 * Asynchronous on ``stream``.  Errors: BBP_EINVAL for bad arguments,
 * algorithm other than BBP_ALG_FUSED or k > 4; BBP_ENOSPACE; BBP_ECUDA.
 */
int bbp_decode_warm(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm, float alpha,
                    double* logp, double* delta, int32_t* iters, int32_t* flags, int8_t* decision, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * bbp_decode_warm_host -- bbp_decode_warm with HOST syndromes and outputs:
 * copies the syndromes in, runs every step above on the device, copies the
 * outputs back and synchronises ``stream`` before returning.  theta and
 * workspace are device memory; the workspace holds at least
 * bbp_decode_warm_workspace_bytes(prm, B, 1) bytes.  Any output pointer
 * except decision may be NULL to skip its copy.  Errors as bbp_decode_warm.
 */
int bbp_decode_warm_host(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm, float alpha,
                         double* logp, double* delta, int32_t* iters, int32_t* flags, int8_t* decision,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Device scratch of bbp_decode_warm (include_io = 0) or bbp_decode_warm_host
 * (include_io != 0) for B syndromes.  Errors: BBP_EINVAL. */
int bbp_decode_warm_workspace_bytes(const bbp_params* prm, int64_t B, int include_io, size_t* bytes);

/*
 * bbp_decode_mixed -- syndromes of different distances in one persistent
 * launch (fused path).  CTAs take (syndrome, coset) items from a counter in
 * ``order`` (e.g. largest distance first); outputs are indexed by syndrome.
 *   syndromes  device, packed: syndrome b starts at byte offsets[b] and has
 *              m(d_of[b]) = 2 d (d-1) bytes
 *   offsets    device [B] int64;  d_of  device [B] int32 (2 <= d <= d_max;
 *              the kernel checks it: a syndrome outside that range is not
 *              decoded, its rows get BBP_FLAG_CHECK and NaN)
 *   order      device [B] int32 permutation of 0..B-1, or NULL (natural order;
 *              an entry outside 0..B-1 is skipped)
 *   prm        k, p, eta, delta0, delta1, max_iter, precision; d is ignored;
 *              algorithm must be BBP_ALG_FUSED; launch_messages = 3 asks for
 *              the register-form-only kernels: the caller vouches that every
 *              distance is odd (k = 4, d_max odd, else BBP_EUNSUPPORTED); a
 *              syndrome of even distance in such a batch gets
 *              BBP_FLAG_CAPACITY.  The default never takes them.
 *   workspace  device, at least 256 bytes (the work counter); when the launch
 *              shape keeps its messages in the workspace (always for k = 5,
 *              6), 256 + bbp_workspace_bytes of d_max and B (the slots)
 * Errors as bbp_decode_batch.
 */
int bbp_decode_mixed(const uint8_t* syndromes, const int64_t* offsets, const int32_t* d_of, const int32_t* order,
                     int64_t B, int32_t d_max, const bbp_params* prm, double* logp, double* delta, int32_t* iters,
                     int32_t* flags, int8_t* decision, void* workspace, size_t workspace_bytes, void* stream);

/* Static text for a return code. */
const char* bbp_strerror(int code);

/* Library version string. */
const char* bbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BLOCKBP_H */
