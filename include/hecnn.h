/*
 * hecnn.h -- C ABI of libhecnn, a GB300 (sm_103a) implementation of the
 * ciphertext-by-ciphertext hot path of encrypted CNN inference in which both
 * the images and the model weights are CKKS ciphertexts (Jain, Nandakumar,
 * Ratha, Pankanti, Kumar, "Efficient CNN Building Blocks for Encrypted Data",
 * arXiv 2102.00319).
 *
 * The calls follow the paper's statement of the problem (Sec. "Homomorphic
 * Encryption"): f(x_1..x_d) = D(g([[x_1]]..[[x_d]]), sk).  Three parties
 * (Sec. "Introduction", Fig. 1): the user holds the secret key, the model
 * owner encrypts weights under the user's public key, the cloud evaluates
 * with evaluation keys only.
 *
 * Conventions for every call
 * --------------------------
 * - Return value: HC_OK (0) or a negative HC_ERR_* code; hc_last_error()
 *   gives a message.  Nothing aborts the process.
 * - Out-parameters are written only on HC_OK.  Every returned handle is owned
 *   by the caller and released with the matching hc_*_destroy.  Input
 *   handles are borrowed and never freed by the library.
 * - Handles belong to one context; destroy them before the context.
 * - Work is enqueued on the context's CUDA stream and is asynchronous; calls
 *   that return host data (export, decrypt+decode, hc_sync) synchronise.
 * - Device memory comes from the context's allocator (default: a
 *   stream-ordered pool on the context stream).
 * - Ciphertexts live on the device in evaluation (NTT) form.  Import and
 *   export use COEFFICIENT form: layout [poly][limb][coeff] of uint64
 *   residues in [0, q_limb), limb i over prime q_i; the *_eval calls move
 *   the evaluation-form words in the same layout.
 * - A context is not thread-safe: one host thread at a time.
 */
#ifndef HECNN_H
#define HECNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
enum {
  HC_OK = 0,
  HC_ERR_INVALID = -1,        /* bad argument, size or handle */
  HC_ERR_LEVEL_MISMATCH = -2, /* operands at different levels */
  HC_ERR_SCALE_MISMATCH = -3, /* scales differ by more than 2^-40 relative */
  HC_ERR_NO_KEY = -4,         /* no Galois key for a requested rotation */
  HC_ERR_DEPTH = -5,          /* rescale (or a layer) needs a level that is not left */
  HC_ERR_OOM = -6,            /* allocator returned NULL */
  HC_ERR_CUDA = -7,           /* a CUDA runtime call failed */
  HC_ERR_TIMEOUT = -8         /* a bounded device wait ran out */
};

typedef struct hc_params hc_params;
typedef struct hc_ctx hc_ctx;
typedef struct hc_secret_key hc_sk;  /* user only */
typedef struct hc_public_key hc_pk;  /* user and model owner */
typedef struct hc_eval_keys hc_evk;  /* cloud: relinearisation + Galois keys, no secret */
typedef struct hc_pt hc_pt;          /* plaintext polynomial at a level and scale */
typedef struct hc_ct hc_ct;          /* ciphertext: degree 1 or 2, level, scale */

/* ------------------------------------------------------------ parameters */
/*
 * Ring degree N = 2^log_n (the paper's phi(m) with m = 2N, K = N/2 slots;
 * Sec. "Impact of FHE parameters").  The modulus chain q_0..q_L ("L" in the
 * paper is the total bit size; here it is the number of rescalable primes)
 * and the special primes p_0..p_{alpha-1} of hybrid key switching.  Each
 * prime is the largest unused prime below 2^bits that is 1 mod 2N, chosen in
 * the order q_0, q_1..q_L, p_0..  Key switching uses dnum = ceil((L+1)/alpha)
 * digits of alpha consecutive primes from q_0.
 */
typedef struct hc_params_desc {
  int log_n;          /* 10..16 */
  int n_q;            /* L + 1, 1..60 */
  const int *q_bits;  /* n_q bit sizes, each 20..61 */
  int n_p;            /* alpha, 1..16 */
  const int *p_bits;  /* n_p bit sizes, each 20..61 */
  double log2_scale;  /* default scale Delta = 2^log2_scale */
  double sigma;       /* error standard deviation (3.2); tail cut floor(6 sigma) */
} hc_params_desc;

/* Builds the prime chain and constants (host only).  HC_ERR_INVALID if a
 * size is out of range or a bit size runs out of primes. */
int hc_params_create(const hc_params_desc *desc, hc_params **out);
void hc_params_destroy(hc_params *p);
/* Writes q_0..q_L, p_0..p_{alpha-1} (n_q + n_p words) into out[cap]. */
int hc_params_primes(const hc_params *p, uint64_t *out, int cap);
/* Degree N, L, alpha, dnum. */
int hc_params_info(const hc_params *p, int *n, int *L, int *alpha, int *dnum);
/* The 63-bit cumulative table of the error sampler (tail-cut entries). */
int hc_params_cdt(const hc_params *p, uint64_t *out, int cap);

/* -------------------------------------------------------------- context */
/* Optional allocator: alloc(bytes, stream, user) returns device memory
 * usable on `stream` (or NULL), free(ptr, stream, user) releases it in
 * stream order. */
/* Device memory callbacks.  Returned blocks must be 16-byte aligned (the
 * kernels move limbs in 16-byte vectors); a misaligned block is freed and
 * the call fails with HC_ERR_INVALID. */
typedef struct hc_allocator {
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, void *stream, void *user);
  void *user;
} hc_allocator;

/* Uploads twiddle and basis-conversion tables to `device` and binds the
 * context to `cuda_stream` (a cudaStream_t, NULL = the legacy default
 * stream).  `alloc` may be NULL (built-in stream-ordered pool).  The params
 * object may be destroyed afterwards. */
int hc_ctx_create(const hc_params *p, int device, void *cuda_stream, const hc_allocator *alloc,
                  hc_ctx **out);
void hc_ctx_destroy(hc_ctx *ctx);
/* Blocks until all work enqueued by the context has finished. */
int hc_sync(hc_ctx *ctx);
/* Message of the last failing call on this context ("" if none). */
const char *hc_last_error(const hc_ctx *ctx);
/* Number of kernels this context has launched so far. */
uint64_t hc_kernel_launches(const hc_ctx *ctx);
/* Per-kernel device timing (tracing aid): while enabled, every kernel launch
 * of the context is bracketed by two CUDA events on the context stream.
 * Enabling (on = 1) clears previous records; on = 0 stops recording. */
int hc_profile_enable(hc_ctx *ctx, int on);
/* Launch count, summed device time (ms) and work units of the kernel `name`
 * since the last enable (synchronises).  A unit is one N-coefficient limb of
 * the launch's output domain (NTT passes: limbs transformed; key product:
 * output slots; conversions and combines: output limbs; the tensor
 * accumulation k_tensor_acc: one (term, limb) pair, i.e. N products of
 * two degree-1 ciphertexts' limbs).  Unknown names report zero. */
int hc_profile_kernel(hc_ctx *ctx, const char *name, uint64_t *launches, double *total_ms,
                      uint64_t *units);
/* Names of the kernels recorded, comma separated, into buf[cap]. */
int hc_profile_names(hc_ctx *ctx, char *buf, size_t cap);
/* Timeline of the last hc_mul_relin_rescale_host call on this context: for
 * each pipeline chunk c, out[6c .. 6c+5] = milliseconds
 * from the call's start to the start and end of the chunk's copies in, of
 * its kernels and of its copies out (CUDA events on the three streams).
 * Writes min(count, cap) values (out may be NULL) and returns the count
 * (6 x chunks; 0 before the first such call). */
int hc_profile_host_timeline(const hc_ctx *ctx, double *out, int cap);
/* Integer-multiplier throughput of this GPU (measurement aid; the paper has
 * no counterpart: its timings are HElib's on CPUs).  Times eight forms,
 * each as four independent dependency chains per thread over 8 blocks of
 * 256 threads per SM: 32-bit multiply-add, 32-bit high half, 32 x 32 -> 64
 * multiply-add, 64-bit low product, 64-bit high product, 64 x 64 -> 128
 * multiply-accumulate with carry (the tensor sums' step), lazy Shoup
 * product by a constant, Harvey's lazy Cooley-Tukey butterfly (the NTT's
 * step), and the epilogue of a split-integer (tensor-core) basis
 * conversion per output residue: 15 fp32 partial sums to integers, their
 * 128-bit assembly and its reduction.  rates[0..8] receive operations per
 * SM per clock at the device's maximum SM clock, rates[9..17] operations
 * per second.  cap < 18 gives HC_ERR_INVALID.  Uses a small buffer from the context allocator and
 * synchronises the context stream.  The roofline of the modular arithmetic
 * (NTT butterflies, tensor accumulation) is derived from these rates. */
int hc_int_mul_rates(hc_ctx *ctx, double *rates, int cap);

/* ----------------------------------------------------------------- keys */
/*
 * Key generation from one 64-bit seed (Philox4x64-10 counter streams, key =
 * (seed, domain tag)): secret s uniform ternary; public key
 * (-a s + e, a) over q_0..q_L; relinearisation key, digit j:
 * (-a_j s + e_j + P [limb in digit j] s^2, a_j) over q_0..q_L, p_0..;
 * a Galois key, same with kappa_g(s) in place of s^2, for every rotation
 * step in rot_steps (left rotation by r uses g = 5^r mod 2N; steps equal
 * mod K share a key; steps = 0 mod K need none).
 */
int hc_keygen(hc_ctx *ctx, uint64_t seed, const int32_t *rot_steps, int n_rot, hc_sk **sk,
              hc_pk **pk, hc_evk **evk);
void hc_sk_destroy(hc_sk *);
void hc_pk_destroy(hc_pk *);
void hc_evk_destroy(hc_evk *);
/* Secret coefficients (int8 values -1, 0, 1) into out[N]. */
int hc_sk_export(hc_ctx *ctx, const hc_sk *sk, int8_t *out, size_t n);
/* Public key, coefficient form: [2][L+1][N] words (b then a). */
int hc_pk_export(hc_ctx *ctx, const hc_pk *pk, uint64_t *out, size_t cap_words);
/* Switching key of rotation `galois_elt` (1 = relinearisation), coefficient
 * form: [dnum][2][L+1+alpha][N] words (b_j then a_j). */
int hc_evk_export(hc_ctx *ctx, const hc_evk *evk, uint64_t galois_elt, uint64_t *out,
                  size_t cap_words);

/* ------------------------------------------------ plaintext / ciphertext */
/* Canonical-embedding encoding (Sec. "Convolution Operator": slot k holds
 * value k): m_i = round(scale (2/N) Re sum_j z_j zeta^{-5^j i}), computed by
 * an FFT in FP64 on the host; n <= K values (the rest zero); im may be NULL.
 * level in 0..L. */
int hc_encode(hc_ctx *ctx, const double *re, const double *im, size_t n, double scale, int level,
              hc_pt **out);
/* Integer plaintext from signed coefficients (|c| < 2^62), N of them. */
int hc_pt_from_coeffs(hc_ctx *ctx, const int64_t *coeffs, size_t n, int level, double scale,
                      hc_pt **out);
/* Coefficient-form residues [level+1][N]. */
int hc_pt_export(hc_ctx *ctx, const hc_pt *pt, uint64_t *out, size_t cap_words);
/* Slots of a plaintext: centred CRT lift, then z_j = scale^{-1} m(zeta^{5^j}). */
int hc_decode(hc_ctx *ctx, const hc_pt *pt, double *re, double *im, size_t n);
int hc_pt_level(const hc_pt *pt);
double hc_pt_scale(const hc_pt *pt);
void hc_pt_destroy(hc_pt *);

/* Public-key encryption (the model owner encrypts weights with the user's
 * public key, Sec. "Introduction"): v ternary, e0, e1 Gaussian from streams
 * (seed, tag of nonce); ct = (v b + e0 + m, v a + e1) at the plaintext's
 * level.  nonce < 2^61; one (seed, nonce) per ciphertext. */
int hc_encrypt(hc_ctx *ctx, const hc_pk *pk, const hc_pt *pt, uint64_t seed, uint64_t nonce,
               hc_ct **out);
/* m = c0 + c1 s (+ c2 s^2) at the ciphertext's level. */
int hc_decrypt(hc_ctx *ctx, const hc_sk *sk, const hc_ct *ct, hc_pt **out);

/* Metadata of a ciphertext in host form. */
typedef struct hc_ct_meta {
  int level;   /* limbs = level + 1 */
  int degree;  /* 1 or 2 (polys = degree + 1) */
  double scale;
} hc_ct_meta;
/* Coefficient-form export, [degree+1][level+1][N] words (synchronises). */
int hc_ct_export(hc_ctx *ctx, const hc_ct *ct, uint64_t *out, size_t cap_words, hc_ct_meta *meta);
/* Import from the same layout; residues must be < q (else HC_ERR_INVALID). */
int hc_ct_import(hc_ctx *ctx, const uint64_t *host, const hc_ct_meta *meta, hc_ct **out);
/* Batched import of n ciphertexts (host[i] with metas[i]): one copy per
 * ciphertext, one range check and one synchronisation for the batch; on any
 * residue >= q nothing is returned (HC_ERR_INVALID). */
int hc_ct_import_batch(hc_ctx *ctx, const uint64_t *const *host, const hc_ct_meta *metas, int n, hc_ct **out);
/* Batched export: one inverse NTT launch for all, asynchronous copies into
 * host[i] (capacity cap[i] words), one synchronisation. */
int hc_ct_export_batch(hc_ctx *ctx, const hc_ct *const *cts, int n, uint64_t *const *host, const size_t *cap);
/* Evaluation-form export and import: the device words as they are (each
 * limb the negacyclic NTT of the residue polynomial, slot k holding the
 * value at psi^(2 brv(k) + 1)), the same [degree+1][level+1][N] layout, no
 * transform.  The form in which a client that computes in evaluation form
 * hands ciphertexts over; import range-checks (residue >= q: HC_ERR_INVALID).
 * Export synchronises. */
int hc_ct_export_eval(hc_ctx *ctx, const hc_ct *ct, uint64_t *out, size_t cap_words, hc_ct_meta *meta);
int hc_ct_import_eval(hc_ctx *ctx, const uint64_t *host, const hc_ct_meta *meta, hc_ct **out);
int hc_ct_meta_of(const hc_ct *ct, hc_ct_meta *meta);
void hc_ct_destroy(hc_ct *);

/* ----------------------------------------------------------- arithmetic */
/* CT-CT add / sub (Sec. "Convolution Operator": "CT-CT add"): same level
 * and degree, scales equal to 2^-40 relative; result takes x's scale. */
int hc_add(hc_ctx *ctx, const hc_ct *x, const hc_ct *y, hc_ct **out);
int hc_sub(hc_ctx *ctx, const hc_ct *x, const hc_ct *y, hc_ct **out);
/* CT-PT add of the slot constant c: adds round(c * scale) to c0 (Eq. 4's
 * constant term). */
int hc_add_const(hc_ctx *ctx, const hc_ct *x, double c, hc_ct **out);
/* CT-PT mult by the slot constant c encoded at const_scale: every limb times
 * round(c * const_scale); scale multiplies; no rescale (Eq. 4, mean pool). */
int hc_mul_const(hc_ctx *ctx, const hc_ct *x, double c, double const_scale, hc_ct **out);
/* CT-CT mult (Eq. 3): tensor product (a0 b0, a0 b1 + a1 b0, a1 b1) -> degree 2. */
int hc_mul(hc_ctx *ctx, const hc_ct *x, const hc_ct *y, hc_ct **out);
/* Relinearisation by hybrid key switching: ModUp of c2 per digit (fast basis
 * conversion), product with the relinearisation key, ModDown by P.  It is
 * the second half of the paper's CT-CT mult (Sec. "Convolution Operator",
 * Eq. 3: a product of two ciphertexts is again a ciphertext, of the same
 * size, after one multiplicative level); its cost grows with the modulus
 * size like the CT-CT mult timings of Sec. "Impact of FHE parameters". */
int hc_relin(hc_ctx *ctx, const hc_evk *evk, const hc_ct *x, hc_ct **out);
/* Rescale by the last prime: c_i' = (c_i - [c_l]) q_l^{-1} mod q_i, [.]
 * centred; scale /= q_l.  HC_ERR_DEPTH at level 0.  This is the modulus
 * consumed by one multiplicative level (Sec. "Impact of FHE parameters":
 * each added multiplication needs a larger modulus L of a fresh ciphertext;
 * here one prime q_l per level). */
int hc_rescale(hc_ctx *ctx, const hc_ct *x, hc_ct **out);
/* Drops limbs above `level` (scale unchanged): aligns operands that have
 * used different numbers of levels before they are added (the linear and
 * squared terms of Eq. 4's g; the modulus chain of Sec. "Impact of FHE
 * parameters"). */
int hc_drop_to_level(hc_ctx *ctx, const hc_ct *x, int level, hc_ct **out);
/* Left rotation of the slots by `steps` ("rotation of values in the slots",
 * Sec. "Convolution Operator"): kappa_g, g = 5^steps mod 2N, then a key
 * switch from kappa_g(s) to s.  steps = 0 mod K copies. */
int hc_rotate(hc_ctx *ctx, const hc_evk *evk, const hc_ct *x, int steps, hc_ct **out);
/* n rotations of one ciphertext sharing a single ModUp of c1 (the
 * automorphism is applied to the raised digits).  Decrypts like hc_rotate
 * but is not bit-identical to it.  Used by the packing that puts a whole
 * image in one ciphertext (Sec. "Parallelization using multi-threading",
 * last paragraph: single-image latency), where every convolution tap is a
 * rotation of the same ciphertext. */
int hc_rotate_hoisted(hc_ctx *ctx, const hc_evk *evk, const hc_ct *x, const int32_t *steps, int n,
                      hc_ct **outs);
/* n independent CT-CT mult + relin + rescale on pairs (a[k], b[k]), batched
 * into one pass of each kernel. */
int hc_mul_relin_rescale_batch(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *a,
                               const hc_ct *const *b, int n, hc_ct **outs);
/* The same n operations from host memory to host memory.  a_host[k] and
 * b_host[k] hold degree-1 ciphertexts in coefficient form
 * ([2][level+1][N] words, the hc_ct_export layout) at one level >= 1
 * (a_meta/b_meta give level, degree and scale); out_host[k] (capacity
 * out_cap[k] words >= 2 level N) receives the product, rescaled, in the same
 * layout, and out_meta[k] its metadata.  The batch runs as a pipeline of
 * chunks of `chunk` pairs (0: about a sixteenth of n from 32 pairs up,
 * the last of them split into halves, 4 -> 2, 1, 1; an eighth below): copies in, the batched operation and copies out of
 * successive chunks overlap on separate CUDA streams, the chunks' kernels
 * round-robin over HC_TUNE_HOST_STREAMS streams; chunk < 0 gives HC_ERR_INVALID.  The relinearise + rescale tail
 * is formed in coefficient form (one inverse transform per output limb, no
 * forward one), with the same words as hc_mul_relin_rescale_batch followed
 * by hc_ct_export.  Pinned host buffers are needed for the overlap.  Inputs
 * are range-checked on the device; a residue >= its prime gives
 * HC_ERR_INVALID after the call has run, with out_host not valid.  Returns
 * when every output is in host memory.  Not capturable in a graph. */
int hc_mul_relin_rescale_host(hc_ctx *ctx, const hc_evk *evk, const uint64_t *const *a_host,
                              const hc_ct_meta *a_meta, const uint64_t *const *b_host,
                              const hc_ct_meta *b_meta, int n, int chunk, uint64_t *const *out_host,
                              const size_t *out_cap, hc_ct_meta *out_meta);
/* The same host-to-host call with the ciphertexts in evaluation form (the
 * hc_ct_export_eval layout) in and out: no forward transform of the inputs
 * and the device batch's own relinearise + rescale tail, so each output
 * equals hc_mul_relin_rescale_batch's followed by hc_ct_export_eval.  Same
 * arguments, chunking, range check and errors as hc_mul_relin_rescale_host. */
int hc_mul_relin_rescale_host_eval(hc_ctx *ctx, const hc_evk *evk, const uint64_t *const *a_host,
                                   const hc_ct_meta *a_meta, const uint64_t *const *b_host,
                                   const hc_ct_meta *b_meta, int n, int chunk, uint64_t *const *out_host,
                                   const size_t *out_cap, hc_ct_meta *out_meta);
/* The evaluation-form call without waiting for it: the copies and kernels
 * are enqueued (out_meta is written at once), *op receives a handle, and
 * hc_host_op_wait(op) returns when every output is in host memory (with
 * the call's result code: a residue >= its prime gives HC_ERR_INVALID
 * there) and releases the handle.  Several calls on one context may be in
 * flight at once, so that one call's copies in overlap the previous call's
 * last kernels and copies out; host buffers must stay valid and unchanged
 * until their call's wait returns.  chunk = 0 here means eighths of n from
 * 32 pairs up (about n / 8 below).  Each handle is waited for exactly once;
 * destroy the context only after every wait.  The call's timeline
 * (hc_profile_host_timeline) is recorded by its wait. */
typedef struct hc_host_op hc_host_op;
int hc_mul_relin_rescale_host_eval_async(hc_ctx *ctx, const hc_evk *evk, const uint64_t *const *a_host,
                                         const hc_ct_meta *a_meta, const uint64_t *const *b_host,
                                         const hc_ct_meta *b_meta, int n, int chunk, uint64_t *const *out_host,
                                         const size_t *out_cap, hc_ct_meta *out_meta, hc_host_op **op);
int hc_host_op_wait(hc_host_op *op);

/*
 * Relinearisation that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot allocate while they run
 * (device memory fixed at start-up, a serving loop that must not enter the
 * allocator); it calls no cudaMalloc, cudaFree or allocator callback of the
 * context.  Same result as
 * hc_relin, written into `out`, a degree-1 ciphertext at x's level that the
 * caller allocated earlier (for example by hc_ct_import); its contents are
 * overwritten and its scale set to x's.  Scratch comes from one static
 * device array of 2^21 64-bit words (16 MiB) that every GPU loading the
 * library holds until exit; a level whose key switch needs more returns
 * HC_ERR_INVALID with the sizes in hc_last_error.  The first call on a
 * device looks up the array's device address (with that device current):
 * make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents; calls whose work overlaps on
 * the GPU (other streams, other threads) race and must be serialised.
 */
int hc_relin_noalloc(hc_ctx *ctx, const hc_evk *evk, const hc_ct *x, hc_ct *out);

/* ------------------------------------------------------------ autotuning */
/*
 * Tile and launch shapes picked by measurement.  The paper has no
 * counterpart (its CPU code has no tiles); results are bit-identical for
 * every choice, only the speed changes.  Knobs:
 *   HC_TUNE_NTT             NTT form for the context's ring degree:
 *                           two passes through global memory with blocks of
 *                           0 = 256 threads (tiles of 16 columns / rows at
 *                           N = 2^16), 1 = 128 threads (tiles of 8, the
 *                           default), 2 = 64 threads (tiles of 4; N >= 2^13);
 *                           or one pass (N >= 2^13): each limb held in the
 *                           shared memory of a cluster of N / 2^14 CTAs (one
 *                           CTA up to 2^14), the stages across CTAs through
 *                           distributed shared memory, register rounds of up
 *                           to 5 (3) or 4 (4) stages; or 5 = the 128-thread
 *                           two-pass form pipelined (N >= 2^13): as many
 *                           CTAs as are resident at once, each copying its
 *                           next tile into shared memory asynchronously while
 *                           it transforms the current one.  The transforms
 *                           that carry the fused relinearise + rescale tail
 *                           stay two-pass (128-thread tiles under 3, 4, 5);
 *   HC_TUNE_KEY_PRODUCT_Z   item groups of a key-product launch, as a
 *                           multiple (1..64) of the default;
 *   HC_TUNE_MODUP_SPLIT     blocks (1..64) over which a ModUp conversion
 *                           splits its output primes;
 *   HC_TUNE_TENSOR_GROUP    sums of tensor products (conv, FC): 0 = one
 *                           output per thread, g = 1..5 (default 5) = up to
 *                           g outputs sharing their x operands per thread
 *                           (a conv position's channels, an FC's classes),
 *                           each x word loaded once; not timed by
 *                           hc_autotune;
 *   HC_TUNE_HOST_STREAMS    hc_mul_relin_rescale_host: its chunks' kernels
 *                           round-robin over 1..4 streams (default 2: the
 *                           context stream and one more); not timed by
 *                           hc_autotune.
 * hc_autotune times each knob's candidates on scratch data shaped like
 * `items` ciphertext pairs at the top level (one knob at a time, the others
 * at their current values, three timed launches each after a warm-up) and
 * keeps the fastest, unless it is less than 2 % faster than the knob's
 * current value (which then stays).  `report` (may be NULL; cap bytes, always
 * NUL-terminated) receives one line per knob: the chosen value and the
 * microseconds per launch of every candidate.  Not capturable; it
 * synchronises the context stream.
 */
enum { HC_TUNE_NTT = 0, HC_TUNE_KEY_PRODUCT_Z = 1, HC_TUNE_MODUP_SPLIT = 2, HC_TUNE_TENSOR_GROUP = 3,
       HC_TUNE_HOST_STREAMS = 4 };
int hc_autotune(hc_ctx *ctx, const hc_evk *evk, int items, char *report, size_t cap);
int hc_tune_set(hc_ctx *ctx, int knob, int value);
/* The knob's current value, or a negative error code. */
int hc_tune_get(const hc_ctx *ctx, int knob);

/* ------------------------------------------------------- graph capture */
/*
 * One CUDA graph for a whole multi-instance computation, replayed with one
 * launch.  The n contexts (distinct, none on the legacy default stream) may
 * share one CUDA stream or use several: the capture runs on the first
 * context's stream, every other stream joins it at hc_graph_begin and is
 * joined back at hc_graph_end, so work issued on different contexts' streams
 * becomes parallel branches of the graph (ordered as the streams order it).
 * hc_graph_launch runs it on the first context's stream, after the work
 * already issued on every captured context's stream, and makes later work
 * on those streams wait for it, so each context sees the launch in its own
 * stream order (results can be read through any of them).  hc_graph_begin
 * gives each context an arena of
 * arena_bytes device bytes (allocated before capture starts) from which every
 * temporary and every output created until hc_graph_end is carved, so the
 * captured work allocates nothing; small index tables are written by kernels
 * that carry them as parameters.  Only evaluation calls (arithmetic, key
 * switching, layers) may be issued while capturing; calls that synchronise
 * (import, export, encrypt, decrypt, keygen) fail.  Handles created while
 * capturing point into the arenas: each hc_graph_launch overwrites their
 * contents; destroy them before the graph.  HC_ERR_OOM if an arena runs out
 * (the capture is then abandoned by hc_graph_end).
 */
typedef struct hc_graph hc_graph;
int hc_graph_begin(hc_ctx *const *ctxs, int n, size_t arena_bytes);
int hc_graph_end(hc_ctx *const *ctxs, int n, hc_graph **out);
int hc_graph_launch(hc_graph *g);
void hc_graph_destroy(hc_graph *g);

/* ---------------------------------------------------------- CNN layers */
typedef enum hc_packing {
  HC_PACK_BATCH = 0,          /* Fig. 2: one ciphertext per pixel / weight, slot k = image k */
  HC_PACK_SINGLE = 1,         /* whole image row-major in one ciphertext (Sec. "Parallelization",
                                 single-image latency) */
  HC_PACK_SINGLE_HOISTED = 2  /* as HC_PACK_SINGLE, the rotations share one ModUp (conv only) */
} hc_packing;

/*
 * Encrypted convolution, Eq. 3: Y_{m,n} = < X^_{m,n}, W^ > over windows
 * anchored top-left, no padding, stride `stride`.  Every output is the sum
 * of all kh*kw*cin tensor products followed by ONE relinearisation and ONE
 * rescale (one level).
 * HC_PACK_BATCH: x[(h*W + w)*cin + ci] (H*W*cin ciphertexts),
 *   w[((co*kh + p)*kw + q)*cin + ci] (cout*kh*kw*cin slot-constant
 *   ciphertexts), y[(m*Wo + n)*cout + co] with Ho = (H-kh)/stride + 1.
 * HC_PACK_SINGLE: cin = 1, stride = 1, x[0] holds the image row-major with
 *   width W; y[co] = sum_{p,q} rot(x, p*W + q) (x) w[(co*kh + p)*kw + q]
 *   (needs Galois keys for every p*W + q); output (m,n) in slot m*W + n.
 * HC_PACK_SINGLE_HOISTED: the same with hoisted rotations (one ModUp of x
 *   for all kh*kw steps); decrypts alike, not bit-identical to SINGLE.
 * Inputs at one level >= 1 with one scale per operand kind; weights at a
 * higher level are dropped to the inputs' level.
 */
int hc_enc_conv2d(hc_ctx *ctx, const hc_evk *evk, hc_packing packing, const hc_ct *const *x,
                  int H, int W, int cin, const hc_ct *const *w, int cout, int kh, int kw,
                  int stride, hc_ct **y);
/*
 * Single-ciphertext-packed convolution of many images (one ciphertext each,
 * image row-major with width W, cin = 1, stride 1) with one set of
 * cout x kh x kw slot-constant weights:
 *   y[i*cout + co] = sum_{p,q} rot(x[i], p*W + q) (x) w[(co*kh + p)*kw + q],
 * one relinearisation and one rescale per output.  Images may sit at
 * different levels: they are grouped by level and every rotation step runs
 * as one batched key switch per group, the groups concurrently on side
 * streams joined back to the context stream (concurrent branches when
 * captured into a graph); weights at a higher level are dropped to each
 * group's level.  Bit-identical to hc_enc_conv2d with HC_PACK_SINGLE
 * applied image by image.
 */
int hc_enc_conv2d_single_batch(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *x, int nimg, int W,
                               const hc_ct *const *w, int cout, int kh, int kw, hc_ct **y);
/*
 * The same convolution with hoisted rotations: per level group one ModUp of
 * every image's c1, then one key product (reading the raised digits through
 * each step's automorphism), one ModDown and one automorphism of c0 over all
 * (step, image) items.  Bit-identical to hc_enc_conv2d with
 * HC_PACK_SINGLE_HOISTED applied image by image (not to
 * hc_enc_conv2d_single_batch: the two rotation forms round differently).
 * Same arguments and errors as hc_enc_conv2d_single_batch.
 */
int hc_enc_conv2d_single_hoisted_batch(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *x, int nimg, int W,
                                       const hc_ct *const *w, int cout, int kh, int kw, hc_ct **y);

/*
 * Polynomial activation g(u) = c0 + c1 u + c2 u^2 (Eq. 4, the paper's
 * 0.47, 0.50, 0.09 approximation of ReLU; (0,0,1) is x^2), elementwise over
 * n ciphertexts.  x^2 uses one level: rescale(relin(u (x) u)).  The general
 * form uses two: t = rescale(relin(u (x) u)); t = rescale(t * c2 @ q_{l-1});
 * v = rescale(u * c1 @ s_t q_l / s_u) dropped to t's level; out = t + v + c0.
 * degree 7 (coeffs c_0..c_7, e.g. a ReLU interpolant) uses four levels, a
 * Paterson-Stockmeyer split with baby steps u, u^2, u^3 and giant step u^4:
 * u2 = rs(rl(u u)); u4 = rs(rl(u2 u2)); u3 = rs(rl(u2 u));
 * deg3(a) = a0 + a1 u + a2 u2 + a3 u3 at level l-3 with the scale of
 * rs(u3 * a3 @ q_{l-2}) (the u and u2 terms brought to it by their
 * constant's scale); out = rs(rl(deg3(c4..c7) u4)) + rs(deg3(c0..c3) * 1 @ s)
 * with s chosen to match scales.  degree must be 2 or 7.  Degree 2 accepts
 * inputs at several levels (each level's inputs form one batch; the
 * batches run concurrently on side streams joined back to the context
 * stream); degree 7 needs one level.
 */
int hc_enc_poly_act(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *x, int n,
                    const double *coeffs, int degree, hc_ct **y);
/*
 * Mean pooling over non-overlapping 2x2 blocks (Eq. 5-6 with the activation
 * applied first): ((a + b) + (c + d)) * 1/4 @ q_l, rescale (one level).
 * HC_PACK_BATCH: x[(h*W + w)*C + c] -> y[(i*(W/2) + j)*C + c].
 * HC_PACK_SINGLE: x[c] holds channel c row-major with width W (H unused):
 *   y[c] = ((x + rot(x, W)) + (rot(x, 1) + rot(x, W+1))) * 1/4 @ q_l, rescaled,
 *   the three rotations hoisted; pooled (i, j) lands in slot 2i W + 2j.
 */
int hc_enc_pool(hc_ctx *ctx, const hc_evk *evk, hc_packing packing, const hc_ct *const *x, int C,
                int H, int W, hc_ct **y);
/*
 * Fully connected layer Z = W X (+ bias) (Sec. "Convolutional Neural
 * Network"): z_r = rescale(relin(sum_k x_k (x) w[r*n_in + k]) [+ bias_r]).
 * Weights (and bias) at a level >= the activations' are dropped to it.
 * bias may be NULL; if given, its scale must equal scale(x) * scale(w).
 */
int hc_enc_fc(hc_ctx *ctx, const hc_evk *evk, hc_packing packing, const hc_ct *const *x, int n_in,
              const hc_ct *const *w, const hc_ct *const *bias, int n_out, hc_ct **y);
/*
 * The FC layer's sums of tensor products before relinearisation:
 * y[r] = sum_k x_k (x) w[r*n_in + k], degree 2, at the activations' level,
 * scale(x) * scale(w) (HC_PACK_BATCH only).  For the FC split over the
 * filters that the paper's multi-threading assigns to separate threads
 * (Sec. "Parallelization using multi-threading"): each part covers the
 * activations of its own filters; the parts are added (hc_add, exact
 * modular addition) and the sum relinearised and rescaled once (hc_relin,
 * hc_rescale), which gives the words of hc_enc_fc over all inputs.
 */
int hc_enc_fc_partial(hc_ctx *ctx, hc_packing packing, const hc_ct *const *x, int n_in, const hc_ct *const *w,
                      int n_out, hc_ct **y);
/* n relinearisations each followed by a rescale, batched into one pass of
 * each kernel with the rescale fused into ModDown's transform: the second
 * half of the FC (and conv) outputs' CT-CT mult (Eq. 3).  d[k]: degree-2
 * ciphertexts at one level >= 1; outs[k] = rescale(relin(d[k])), the same
 * words as hc_rescale(hc_relin(d[k])) and as the tail of hc_enc_fc. */
int hc_relin_rescale_batch(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *d, int n, hc_ct **outs);

/*
 * Fully connected layer on single-ciphertext activations: x[c] (c < C)
 * hold the features of channel c at arbitrary slots; w[r*C + c] holds, in
 * the same slots, the weights of class r for channel c (the model owner
 * encrypts these vectors).  z_r = rs(rl(sum_c x_c (x) w[r*C+c])), then
 * z_r += rot(z_r, 2^k) for k < span_log2: slot 0 of y[r] holds the class
 * score when the features lie in slots below 2^span_log2.  Needs Galois
 * keys for the powers of two; weights above x's level are dropped to it.
 */
int hc_enc_fc_rotsum(hc_ctx *ctx, const hc_evk *evk, const hc_ct *const *x, int C, const hc_ct *const *w,
                     int n_out, int span_log2, hc_ct **y);

#ifdef __cplusplus
}
#endif
#endif /* HECNN_H */
