/*
 * fhe.h -- C ABI of the GB300 (sm_103a) RNS-CKKS hybrid key-switching library.
 *
 * The library implements the key-switching hot path studied in "Theodosian:
 * A Deep Dive into Memory-Hierarchy-Centric FHE Acceleration" (arXiv
 * 2512.18345): INTT -> ModUp BConv -> NTT -> key inner product -> INTT ->
 * ModDown BConv -> NTT (+ combine), Section IV and Fig. "keysw", and the CKKS
 * operations built on it (HMult relinearisation, HRotate, rescale, hoisted
 * rotations, plaintext multiply).  All work runs in hand-written CUDA kernels
 * on one GPU; there is no CPU fallback.
 *
 * Data conventions (Section II-A: a polynomial is an L x N matrix of 32-bit
 * residues, row i reduced modulo its own prime):
 *   - polynomial at level l: uint32 [l][N], limb-major, limb i modulo q_i,
 *     every residue fully reduced to [0, q_i), NTT (evaluation) form in
 *     bit-reversed slot order: slot i holds the value at psi^(2 brv(i) + 1);
 *   - ciphertext: uint32 [2][l][N] = (c0, c1), decrypting as c0 + c1 s;
 *   - switching key: uint32 [dnum][2][L + K][N] = (b_j, a_j) per digit j with
 *     b_j = -a_j s + e_j + g_j s', g_j = [P]_{q_i} on digit j's limbs, 0
 *     elsewhere; rows 0..L-1 are q-limbs, rows L..L+K-1 the special primes;
 *   - digits: alpha = ceil(L / dnum) limbs each, digit j = limbs
 *     [j alpha, min((j + 1) alpha, l)); beta(l) = ceil(l / alpha);
 *   - psi (primitive 2N-th root per prime) = g^((q-1)/2N) for the smallest
 *     integer g >= 2 with psi^N = -1 (mod q).
 *
 * Pointers: polynomial, ciphertext and output arguments are DEVICE pointers
 * owned by the caller, 16-byte aligned, on the context's device.  Key and
 * prime-list arguments may be host or device pointers (copied).  Outputs must
 * not overlap inputs unless a function says so (FHE_EALIAS otherwise).
 *
 * Streams: every call is asynchronous on the given stream (a cudaStream_t,
 * e.g. torch.cuda.Stream().cuda_stream; 0 = legacy default stream).  A
 * context owns one scratch workspace; consecutive calls on one context are
 * ordered by the library even across different streams (each call waits for
 * the previous call's stream through an event), so calls on one context never
 * run concurrently.  Use one context per concurrent stream.
 *
 * Errors: every function returns FHE_OK (0) or a negative status; argument
 * errors are detected on the host before anything is enqueued.  The library
 * never prints, exits or throws.  fhe_last_error() returns a thread-local
 * message for the last non-OK status.
 */
#ifndef FHE_GB300_H
#define FHE_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(FHE_BUILD)
#define FHE_API __attribute__((visibility("default")))
#else
#define FHE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FHE_OK 0
#define FHE_EINVAL (-1)       /* bad argument (null pointer, size, alignment, count) */
#define FHE_ELEVEL (-2)       /* level outside [1, L] (or < 2 for rescale) */
#define FHE_ENOKEY (-3)       /* the needed switching key was never set */
#define FHE_EPRIME (-4)       /* a prime is not prime, not 1 mod 2N, >= 2^31, <= 2^20, or repeated */
#define FHE_ENOMEM (-5)       /* device allocation failed */
#define FHE_ECUDA (-6)        /* a CUDA runtime call failed (message in fhe_last_error) */
#define FHE_EALIAS (-7)       /* output overlaps an input */
#define FHE_ETIMEOUT (-8)     /* a bounded device-side wait expired */
#define FHE_EUNSUPPORTED (-9) /* valid but not supported (e.g. N outside 2^12..2^16) */

#define FHE_MAX_PRIMES 64
#define FHE_RELIN_KEY INT32_MIN /* key_id of the relinearisation key in fhe_keyswitch */

typedef struct fhe_ctx fhe_ctx;
typedef struct fhe_plan fhe_plan;
typedef void *fhe_stream;

typedef struct {
  uint32_t N;
  int L, K, dnum, alpha;
  int device;
  size_t limb_bytes;      /* 4 N */
  size_t key_bytes;       /* dnum * 2 * (L + K) * limb_bytes, one switching key */
  size_t workspace_bytes; /* device scratch the context owns */
  size_t table_bytes;     /* device twiddle / base-conversion tables */
  int n_rot_keys;         /* rotation keys currently set */
  int bconv_mode;         /* FHE_BCONV_SCALAR or FHE_BCONV_TC */
  uint32_t psi[FHE_MAX_PRIMES]; /* psi of q_0..q_{L-1}, p_0..p_{K-1} */
} fhe_info;

/* BConv implementation selector (fhe_ctx_set_bconv).  Both give identical bits. */
#define FHE_BCONV_SCALAR 0 /* CUDA-core 64-bit multiply-accumulate, one final reduction */
#define FHE_BCONV_TC 1     /* tensor cores: 8-bit digit split, f16 operands, exact fp32 accumulation;
                              needs alpha <= 12 and K <= 12 (fhe_bconv: n_in <= 12) */

/*
 * Create a context for ring degree N (a power of two, 2^12..2^16), ciphertext
 * primes q[0..L) and special primes p[0..K) (host pointers), dnum digits, on
 * CUDA device `device`.  Validates the primes (FHE_EPRIME), computes psi per
 * prime and every device table (twiddles with their Shoup companions, the
 * base-conversion tables of Section III-C for every digit and for ModDown,
 * the rescale constants) and allocates the workspace for one key switch at
 * level L.  *out is NULL on error.
 */
FHE_API int fhe_ctx_create(fhe_ctx **out, uint32_t N, const uint32_t *q, int L, const uint32_t *p, int K, int dnum,
                   int device);
FHE_API int fhe_ctx_destroy(fhe_ctx *ctx);
FHE_API int fhe_ctx_info(const fhe_ctx *ctx, fhe_info *out);
/* Select the BConv implementation for later calls (FHE_BCONV_SCALAR / FHE_BCONV_TC).
 * The tensor-core digit split is exact for at most 12 inputs per conversion: a
 * K = 48 contraction when alpha and K are at most 8, a K = 64 one (signed offset
 * pieces) when they are at most 12.  FHE_EUNSUPPORTED for FHE_BCONV_TC when alpha
 * > 12 or K > 12. */
FHE_API int fhe_ctx_set_bconv(fhe_ctx *ctx, int mode);
/*
 * Synchronize the context's device and report device-side failures: returns
 * FHE_ETIMEOUT (and clears the condition) when a kernel's bounded wait on the
 * tensor cores expired since the last call; its outputs are then invalid.
 */
FHE_API int fhe_ctx_sync(fhe_ctx *ctx);
/*
 * Failure-detection self-test (no counterpart in the paper): enqueues one CTA
 * that waits, with the library's bounded wait and a short limit, on a barrier
 * nothing arrives on; the expiry is recorded in the context's status word as a
 * production kernel records it, so the next fhe_ctx_sync returns FHE_ETIMEOUT
 * (and clears it).  No fault, trap or unbounded wait is involved.
 */
FHE_API int fhe_selftest_wait_timeout(fhe_ctx *ctx, fhe_stream stream);
/* Cap the device memory the context may still grow into (workspace slots, the
 * linear transforms' scratch, switching-key copies), in bytes; 0 (the default)
 * removes the cap.  A call that would grow past it returns FHE_ENOMEM before
 * allocating or launching anything, and the context stays usable (memory already
 * held is kept).  Also the host-side way to inject allocation failures in tests. */
FHE_API int fhe_ctx_set_memory_limit(fhe_ctx *ctx, size_t bytes);
/* Fuse stage epilogues (1, default) or run the plain per-kernel pipeline (0).  Same bits. */
FHE_API int fhe_ctx_set_fused(fhe_ctx *ctx, int fused);
/* Complementary pipelining (Section IV-B) in the fused pipeline: with `on`
 * (the default) the inner product of the ciphertext limbs runs on an
 * auxiliary branch beside ModDown's special-limb chain; without it, one launch
 * covers all limbs.  Results are identical either way; fhe_autotune sets it. */
FHE_API int fhe_ctx_set_pipelining(fhe_ctx *ctx, int on);
/* NTT kernel variants (flags; 0 = the two-pass kernels, the default):
 *   FHE_NTT_OTF: the block passes (the last eight stages, the paper's second
 *     NTT kernel, Section III-C) form most of their register twiddles on the fly
 *     from one loaded twiddle and a staged 8-entry table instead of loading each;
 *   FHE_NTT_SINGLE_PASS: each 2^16-point transform of a stage program runs as
 *     one launch with a cluster of 16 CTAs per limb, the first pass's tiles
 *     staying in shared memory for the second (no global round trip);
 *   FHE_NTT_STREAM: the column and block passes run as persistent kernels: a
 *     producer warp copies each tile into a ring of shared-memory stages ahead
 *     of eight consumer warps, which keep their twiddles in registers across
 *     consecutive tiles of the same prime (N = 2^16; the gather, reduce and
 *     rescale forms keep the two-pass kernels).  With FHE_NTT_SINGLE_PASS, the
 *     transforms the single-pass kernel covers use it and the others stream;
 *   FHE_NTT_PERSIST: the transforms the single-pass kernel covers run as one
 *     persistent, cooperative launch each (every CTA resident): the CTAs walk
 *     the first pass's tiles, meet at a grid-wide barrier (bounded; an expired
 *     wait sets status bit 4 and fhe_ctx_sync reports FHE_ETIMEOUT as for
 *     the other waits), then walk the second pass's tiles; the global round
 *     trip stays, the second launch's ramp and the first one's tail go
 *     (N = 2^16; combines with no other flag).
 * Results are identical in every mode.  Programs and plans built after the call
 * use the new mode.  FHE_EUNSUPPORTED for FHE_NTT_STREAM or FHE_NTT_PERSIST at
 * N != 2^16, for FHE_NTT_SINGLE_PASS at N != 2^16 or on a device that cannot
 * hold a 16-CTA cluster of the kernel; FHE_EINVAL for unknown flags and for
 * FHE_NTT_PERSIST with another flag.  fhe_autotune with FHE_TUNE_NTT measures
 * the modes. */
#define FHE_NTT_OTF 1
#define FHE_NTT_SINGLE_PASS 2
#define FHE_NTT_STREAM 4
#define FHE_NTT_PERSIST 8
FHE_API int fhe_ctx_set_ntt(fhe_ctx *ctx, int flags);

/* Kernel shapes (results are identical for every shape; fhe_autotune with
 * FHE_TUNE_SHAPE measures them):
 *   fuse_ip_moddown: 1 runs the key inner product of the K special limbs and
 *     the first pass of ModDown's inverse NTT as one kernel (Section IV,
 *     stage 2 feeding stage 3): u's special limbs stay in registers; for key
 *     switches whose digits are read directly (not hoisted rotations), N = 2^16
 *     and at most four digits;
 *   bconv_tc_ctas: resident CTAs per SM of the tensor-core BConv (1..4; fewer
 *     leave shared memory and tensor memory to kernels of other lanes);
 *   bconv_tc_pipeline: 1 gives each tensor-core BConv CTA two operand buffers
 *     and two tensor-memory accumulators, so that a tile's MMA runs while the
 *     previous tile's accumulator is reduced (at most two CTAs per SM for more
 *     than 16 outputs, one for more than 32);
 *   ntt_stream_stages, ntt_stream_ctas: shared-memory stages per CTA (2..3) and
 *     persistent CTAs per SM (1..3) of the FHE_NTT_STREAM passes;
 *   ip_staged_gather: 1 (the default) has the hoisted inner product (digits
 *     read through an automorphism, Section V-C) copy each digit's permuted
 *     32-coefficient blocks into shared memory with bulk copies, so that every
 *     digit value is a shared-memory read; 0 gathers them with 4-byte global
 *     loads.  Launches that add the pass-through polynomial to both halves
 *     (relinearisation) use the gathering kernel either way;
 *   ip_staged_ctas, ip_staged_depth: resident CTAs per SM (1: one CTA of up
 *     to 227 KB of shared memory; 2: two of up to 113 KB) and stages per warp
 *     (2..4; 0: 2) of that staged kernel, whose warps each run their own
 *     pipeline; a CTA has as many warps as its shared memory holds, at most
 *     16 per SM.
 * Programs and plans built after the call use the new shape.  FHE_EINVAL for a
 * value out of range; FHE_EUNSUPPORTED for fuse_ip_moddown at N != 2^16. */
typedef struct {
  int fuse_ip_moddown;
  int bconv_tc_ctas;
  int ntt_stream_stages;
  int ntt_stream_ctas;
  int bconv_tc_pipeline;
  int ip_staged_gather;
  int ip_staged_ctas;
  int ip_staged_depth;
} fhe_kernel_shape;
FHE_API int fhe_ctx_set_kernel_shape(fhe_ctx *ctx, const fhe_kernel_shape *shape);
FHE_API int fhe_ctx_get_kernel_shape(const fhe_ctx *ctx, fhe_kernel_shape *out);

/*
 * Switching keys ([dnum][2][L + K][N] uint32, NTT form, host or device
 * pointer).  The context copies the key (it owns the copy); the copy is
 * enqueued on `stream`.  A rotation key is stored under its Galois element
 * 5^rot mod 2N, so rot and rot + N/2 share one key.  Setting a key again
 * replaces it.
 */
FHE_API int fhe_set_relin_key(fhe_ctx *ctx, const uint32_t *key, fhe_stream stream);
FHE_API int fhe_set_rot_key(fhe_ctx *ctx, int32_t rot, const uint32_t *key, fhe_stream stream);

/*
 * Hybrid key switching of d ([level][N], NTT form) with the relinearisation
 * key (key_id = FHE_RELIN_KEY) or the rotation key of index key_id (Section
 * IV, Fig. "keysw"): out = (out_0, out_1) [2][level][N] with
 * out_0 + out_1 s = d s' + small.  ModDown is floor type.
 */
FHE_API int fhe_keyswitch(fhe_ctx *ctx, const uint32_t *d, int level, int32_t key_id, uint32_t *out, fhe_stream stream);

/*
 * HRotate: ct [2][level][N] -> out [2][level][N], rotation of the slots by
 * rot (new slot j = old slot j + rot): with k = 5^rot mod 2N,
 * out = (sigma_k(c0) + KS(sigma_k(c1))_0, KS(sigma_k(c1))_1).  The
 * automorphism is applied in NTT form inside the first kernels (Section II-B,
 * "The rest": automorphism is index math).  rot = 0 (mod N/2) copies.
 */
FHE_API int fhe_rotate(fhe_ctx *ctx, const uint32_t *ct, int level, int32_t rot, uint32_t *out, fhe_stream stream);

/*
 * HMult with relinearisation: a, b [2][level][N] -> out [2][level][N]:
 * (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1), out = (d0, d1) + KS(d2).
 * No rescale (call fhe_rescale).
 */
FHE_API int fhe_hmult(fhe_ctx *ctx, const uint32_t *a, const uint32_t *b, int level, uint32_t *out, fhe_stream stream);

/*
 * Floor rescale: ct [2][level][N] -> out [2][level-1][N],
 * out_i = (c_i - NTT_{q_i}(INTT_{q_last}(c_last))) q_last^-1 mod q_i.
 */
FHE_API int fhe_rescale(fhe_ctx *ctx, const uint32_t *ct, int level, uint32_t *out, fhe_stream stream);

/*
 * Hoisted rotations of one ciphertext by rots[0..n): one shared ModUp of c1,
 * then per rotation sigma_k applied to the extended digits (a permutation in
 * NTT form), the inner product with that rotation's key, ModDown and the
 * addition of sigma_k(c0).  outs[i] is a device pointer to [2][level][N].
 * A rotation by 0 copies ct.
 */
FHE_API int fhe_rotate_hoisted(fhe_ctx *ctx, const uint32_t *ct, int level, const int32_t *rots, int n,
                       uint32_t *const *outs, fhe_stream stream);

/*
 * Baby-step / giant-step plaintext matrix-vector product, the linear-transform
 * shape of bootstrapping (hoisted rotations, Section V-C):
 *   out = sum_{g < giant} rot_{baby g}( sum_{b < baby} diags[g baby + b] (.) rot_b(ct) )
 * ct [2][level][N]; diags [giant * baby][level][N] NTT-form plaintexts (device);
 * out [2][level][N] (must not overlap ct).  The baby rotations share one ModUp
 * (as fhe_rotate_hoisted); the giant rotations are ordinary rotations.  Needs the
 * rotation keys of 1..baby-1 and baby g (g = 1..giant-1).  baby <= 32, giant <= 16.
 * No rescale.  The context grows a scratch buffer of (baby + 2 giant) ciphertexts.
 */
FHE_API int fhe_linear_transform(fhe_ctx *ctx, const uint32_t *ct, int level, const uint32_t *diags, int baby,
                                 int giant, uint32_t *out, fhe_stream stream);

/*
 * Double-hoisted baby-step / giant-step transform, the form of the CoeffToSlot /
 * SlotToCoeff levels of bootstrapping (radix-merged FFT levels with few nonzero
 * diagonals; the hoisting literature cited in Section V-C):
 *   out = sum_{g < n_giant} rot_{giant[g]}( sum_{b < n_baby} diags[idx[g n_baby + b]] (.) rot_{baby[b]}(ct) )
 * Every baby rotation shares one ModUp of c1 and stays in the extended basis
 * Q_level u P (no ModDown); the inner sums are formed there; the c1 half of
 * each rotating giant step's inner sum is brought down to Q_level, decomposed
 * again and key-switched, still without ModDown; one ModDown of both halves
 * ends the transform.  Bit-exact against that sequence of exact RNS steps.
 *   ct     [2][level][N] NTT form, device, 16-byte aligned;
 *   baby   [n_baby], giant [n_giant] rotation indices (host); one whose Galois
 *          element is 1 (0 mod N/2) is the identity and needs no key, every other
 *          one needs its rotation key; n_baby <= 32, n_giant <= 16;
 *   diags  [n_diag][level+K][N] NTT-form plaintexts over q_0..q_{level-1} and
 *          p_0..p_{K-1} (device; the extended basis, since they multiply
 *          extended-basis rotations);
 *   idx    [n_giant][n_baby] (host) index into diags, or -1 where the pair has
 *          no diagonal;
 *   out    [2][level][N] (device), must not overlap ct or diags.
 * No rescale.  The context grows a scratch buffer of (n_baby + 2 n_giant + 1)
 * extended-basis ciphertexts plus n_giant polynomials.  Errors: FHE_EINVAL (null,
 * misaligned, counts or idx out of range, n_diag > 32767), FHE_ELEVEL, FHE_ENOKEY, FHE_EALIAS,
 * FHE_ENOMEM, FHE_ECUDA.
 */
FHE_API int fhe_linear_transform_dh(fhe_ctx *ctx, const uint32_t *ct, int level, const int32_t *baby, int n_baby,
                                    const int32_t *giant, int n_giant, const uint32_t *diags, int n_diag,
                                    const int32_t *idx, uint32_t *out, fhe_stream stream);

/* Plaintext multiply: out_c = ct_c * pt ([level][N] NTT form), c = 0, 1. out may equal ct. */
FHE_API int fhe_pmult(fhe_ctx *ctx, const uint32_t *ct, const uint32_t *pt, int level, uint32_t *out, fhe_stream stream);
/* Addition of two [npoly][level][N] arrays (npoly = 2 for ciphertexts). out may equal a or b. */
FHE_API int fhe_add(fhe_ctx *ctx, const uint32_t *a, const uint32_t *b, int npoly, int level, uint32_t *out,
            fhe_stream stream);

/*
 * Stage-level entry points (the individual steps of Fig. "keysw"; used by the
 * parity tests and by callers composing their own pipelines).
 *   fhe_ntt / fhe_intt: in-place transform of n limbs whose primes are
 *     prime_idx[0..n) (indices into q_0..q_{L-1}, p_0..p_{K-1}; host array).
 *   fhe_modup: d [level][N] (NTT form) -> ext [beta][level + K][N] (NTT form),
 *     digit j's own limbs copied from d.
 *   fhe_moddown: u [level + K][N] (NTT form, extended basis) -> out [level][N].
 *   fhe_bconv: coefficient-form fast base conversion of in [n_in][N] (primes
 *     in_idx) to out [n_out][N] (primes out_idx), Section II-B "BConv" with the
 *     table T[i][j] = (Qstar / q_j) mod p_i of Section III-C and the
 *     [(Qstar / q_j)^-1]_{q_j} pre-multiplication; n_in <= 16, n_out <= 64
 *     (n_in <= 12 under FHE_BCONV_TC, else FHE_EUNSUPPORTED).  The context
 *     keeps the tables of each (in_idx, out_idx, kernel) combination: the
 *     first call with a combination allocates them (a few KB) and copies them
 *     on `stream`, and the context's first fhe_bconv call allocates its
 *     [16][N]-word pre-multiplied input; a call with a known combination
 *     allocates nothing and does not synchronize.  At most 64 combinations are
 *     kept: a new one beyond that waits for `stream` and releases them.
 */
FHE_API int fhe_ntt(fhe_ctx *ctx, uint32_t *a, const int *prime_idx, int n, fhe_stream stream);
FHE_API int fhe_intt(fhe_ctx *ctx, uint32_t *a, const int *prime_idx, int n, fhe_stream stream);
FHE_API int fhe_modup(fhe_ctx *ctx, const uint32_t *d, int level, uint32_t *ext, fhe_stream stream);
FHE_API int fhe_moddown(fhe_ctx *ctx, const uint32_t *u, int level, uint32_t *out, fhe_stream stream);
FHE_API int fhe_bconv(fhe_ctx *ctx, const uint32_t *in, const int *in_idx, int n_in, uint32_t *out, const int *out_idx,
              int n_out, fhe_stream stream);

/*
 * Batched key switching (Section IV-A multi-polynomial caching and batching,
 * Section IV-C CUDA Graphs): a plan holds a list of independent operations
 * at uneven levels (at least one); fhe_batch_plan validates them (levels, keys, buffers
 * non-null and 16-byte aligned: FHE_EINVAL; an output overlapping its item's
 * input: FHE_EALIAS), sizes the item groups (fhe_ctx_set_batch,
 * fhe_autotune) and captures the whole batch into one CUDA graph;
 * fhe_batch_launch replays it on `stream`.  Every item's result is
 * bit-identical to the same operation run alone.  The buffers named by the
 * items must stay valid while the plan is used.
 */
#define FHE_OP_KS 0     /* out = KS(in) with key_id = rot (FHE_RELIN_KEY or a rotation index) */
#define FHE_OP_ROTATE 1 /* out = HRotate(in, rot) */
#define FHE_OP_RELIN 2  /* out = HMult(in, in2) with relinearisation */
typedef struct {
  int op;
  int level;
  int32_t rot;
  const uint32_t *in;
  const uint32_t *in2;
  uint32_t *out;
} fhe_ks_item;

#define FHE_PLAN_GRAPH 1 /* capture into a CUDA graph (otherwise launch kernels directly) */
FHE_API int fhe_batch_plan(fhe_ctx *ctx, const fhe_ks_item *items, int n, int flags, fhe_plan **out);
FHE_API int fhe_batch_launch(fhe_plan *plan, fhe_stream stream);
FHE_API int fhe_plan_destroy(fhe_plan *plan);
/* number of kernel launches one fhe_batch_launch performs (graph nodes or direct launches) */
FHE_API int fhe_plan_kernel_count(const fhe_plan *plan);
/* sizes of the plan's item groups (at most max written); returns the number of groups */
FHE_API int fhe_plan_groups(const fhe_plan *plan, int *sizes, int max);
/*
 * Group sizing of later plans: the stage-1 working sets (beta(l)(l+K) limbs per
 * item) of the groups resident at once stay within l2_budget_bytes (0: twice
 * the device's L2), a group holds at most max_group items (0: 8), and groups
 * run round-robin on `lanes` concurrent streams (0: 2), each lane with its own
 * workspace, so that one group's DRAM-bound inner product overlaps another
 * group's transforms.  fhe_autotune measures and sets these.
 */
FHE_API int fhe_ctx_set_batch(fhe_ctx *ctx, size_t l2_budget_bytes, int max_group, int lanes);

/*
 * Schedule autotuner (Section IV-A batching, Section IV-C graphs): measures
 * graph-captured plans of n_items (1..64) synthetic key switches at `level`
 * on `stream` for every candidate schedule -- lanes 1..4, group budgets of
 * 3/4, 1, 2 and 4 times the device's L2, one or two resident CTAs per SM for
 * the streaming inner product (one leaves room for transforms beside it; it is
 * chosen only when more than 2 % faster than the best two-CTA schedule),
 * complementary pipelining (Section IV-B) on or off, and,
 * with FHE_TUNE_BCONV, both BConv kernels -- applies the fastest to the
 * context (fhe_ctx_set_batch, the inner product's residency and, with
 * FHE_TUNE_BCONV, fhe_ctx_set_bconv) and describes it in *out.  Allocates and
 * frees its own buffers; without a relinearisation key it installs a filler
 * key for the run and removes it.  Synchronizes the device.  FHE_EINVAL while
 * `stream` is capturing; FHE_ETIMEOUT if a bounded device wait expired (the
 * context's settings are then left as they were).
 */
#define FHE_TUNE_BCONV 1 /* also choose between the CUDA-core and tensor-core BConv */
#define FHE_TUNE_NTT 2   /* then also measure the NTT variants (fhe_ctx_set_ntt) under the chosen schedule */
#define FHE_TUNE_SHAPE 4 /* then also measure kernel shapes (fhe_ctx_set_kernel_shape) one parameter at a time */
typedef struct {
  int lanes;              /* chosen lane count */
  size_t l2_budget_bytes; /* chosen group budget */
  int max_group;          /* chosen group cap (0: default) */
  int bconv_mode;         /* chosen BConv kernel */
  int n_groups;           /* groups of the measured plan */
  double us_per_ks;       /* measured time per key switch of the chosen schedule, microseconds */
  double default_us_per_ks; /* the same for the default schedule (2 lanes, 2 x L2, 2 CTAs), 0 if not measured */
  int candidates;         /* distinct schedules measured */
  int ip_ctas_per_sm;     /* chosen residency of the streaming inner product */
  int comp_pipe;          /* 1: complementary pipelining (q-limb inner product on its own branch) */
  int ntt_mode;           /* chosen fhe_ctx_set_ntt flags (with FHE_TUNE_NTT; else the context's) */
  fhe_kernel_shape shape; /* chosen kernel shape (with FHE_TUNE_SHAPE; else the context's) */
} fhe_tune_result;
FHE_API int fhe_autotune(fhe_ctx *ctx, int level, int n_items, int flags, fhe_tune_result *out, fhe_stream stream);
/*
 * fhe_autotune with a cache file at `path` (a text file, one line per entry):
 * an entry for this context's (N, level, K, alpha, dnum), n_items, flags and
 * GPU (name and SM count) is applied without measuring (out->candidates = 0);
 * otherwise the schedules are measured as by fhe_autotune and the choice is
 * appended to the file.  Malformed lines are skipped; the last matching entry
 * wins.  FHE_EINVAL if the file cannot be appended to.
 */
FHE_API int fhe_autotune_cached(fhe_ctx *ctx, const char *path, int level, int n_items, int flags,
                                fhe_tune_result *out, fhe_stream stream);

/*
 * Kernel tracing (measurement support): while enabled, every kernel the
 * context launches outside a captured plan is bracketed by two CUDA events on
 * its stream, and the auxiliary branch of complementary pipelining runs on the
 * main stream, so that each interval holds its kernel alone.  fhe_trace_read synchronizes the device, returns per-kernel-name
 * launch counts and summed event times (at most `max` entries, *n = number of
 * distinct names) and clears the record.
 */
typedef struct {
  char name[48];
  int launches;
  double total_ms;
} fhe_kernel_stat;
FHE_API int fhe_trace_enable(fhe_ctx *ctx, int on);
/*
 * Bandwidth probe: read, write and read+write (copy) throughput in GB/s of a
 * `bytes` block accessed `reps` times with 128-bit L2-cached loads and stores
 * on `device` (allocates and frees two blocks).  A block smaller than the L2
 * measures the L2 (the paper's method for its L2 bandwidth figure); the
 * benchmark uses the copy figure as the denominator of its L2-roofline fraction.
 */
FHE_API int fhe_probe_bandwidth(int device, size_t bytes, int reps, double *read_gbs, double *write_gbs,
                                double *copy_gbs);
/*
 * Integer-pipe probe: register-only chains on `device` (four 256-thread CTAs
 * per SM, one wave; allocates and frees a few KB).  Rates are whole-GPU units
 * per second; clock_mhz is the SM clock the chains ran at (cycle counter over
 * event time).  butterflies_per_s is the forward Shoup butterfly exactly as
 * the NTT passes compute it (31-bit prime, values lazily in [0, 2q)): the
 * ALU denominator of the transforms' roofline fractions; mac64_per_s the
 * 32 x 32 -> 64-bit multiply-accumulate of the base conversion.
 */
typedef struct {
  double clock_mhz;
  double butterflies_per_s;
  double mac64_per_s;
  double imad_per_s, imad_hi_per_s, add_min_per_s;
  int sms;
} fhe_int_peaks;
FHE_API int fhe_probe_int(int device, fhe_int_peaks *out);
FHE_API int fhe_trace_read(fhe_ctx *ctx, fhe_kernel_stat *out, int max, int *n);

/*
 * Allocation-free base conversion.  The paper has no counterpart: this entry
 * point is an addition to the interface for callers that cannot allocate
 * device memory once they are running -- a process whose framework has
 * already reserved all free device memory for its own pool (any further
 * cudaMalloc fails), or a real-time loop that must not take cudaMalloc's
 * implicit device-wide synchronization or its unbounded latency.
 *
 * Computes exactly what fhe_bconv computes (same bits, CUDA-core kernel) but
 * allocates nothing: its scratch -- the pre-multiplied input, at most
 * FHE_BCONV_NOALLOC_MAX_IN x FHE_BCONV_NOALLOC_MAX_N words, and the
 * conversion tables -- is one fixed device array of about 2 MB that every GPU
 * loading this library holds until the process exits.  Larger n_in, n_out or
 * N are rejected with FHE_EINVAL (use fhe_bconv).  The context must already
 * exist.  The tables travel to the GPU as kernel arguments, not as copies
 * from host memory.
 *
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents; every word a call reads it writes first, so nothing has to be
 * cleared.  Calls on one context are ordered by the library, but calls whose
 * GPU work overlaps -- unordered streams of different contexts on the same
 * device -- race on the shared array.
 */
#define FHE_BCONV_NOALLOC_MAX_IN 8
#define FHE_BCONV_NOALLOC_MAX_OUT 64
#define FHE_BCONV_NOALLOC_MAX_N 65536
FHE_API int fhe_bconv_noalloc(fhe_ctx *ctx, const uint32_t *in, const int *in_idx, int n_in, uint32_t *out,
                              const int *out_idx, int n_out, fhe_stream stream);

FHE_API const char *fhe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FHE_GB300_H */
