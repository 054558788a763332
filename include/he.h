/*
 * he.h -- C ABI of the GB300 library for the encrypted FFConv layer (arXiv 2102.03494).
 *
 * The library evaluates, on one GPU, the homomorphic FFConv layer of the paper's Sec. 4.2
 * (FFConv packing, DP-HI2C-CP): a d x d low-rank convolution W1 under DensePack (Sec. 3.2,
 * Fig. 1) followed by a 1 x 1 restoring convolution W2 under ConvPack (Sec. 3.2, Fig. 2a),
 * on RNS-BFV ciphertexts (Sec. 2.1: plaintext modulus t, ciphertext modulus Q, ring
 * dimension N).  Every step runs in the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Return value: HE_OK (0) or a negative HE_E* code; he_last_error() gives the message.
 *     Nothing throws across the ABI.
 *   - "device" pointers are CUDA device memory owned by the caller; "host" pointers are
 *     ordinary host memory owned by the caller.  The context owns its tables, its resident
 *     Galois keys and its scratch memory.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous unless stated;
 *     entry points that return data in host memory synchronise that stream.
 *   - A context is not thread-safe; use one per host thread.
 *   - Ring elements are stored limb-major: a ciphertext is [2][n_limbs][N] uint64 residues,
 *     limb i reduced modulo the i-th ciphertext prime.  Slot vectors are N int64 values
 *     (slot j < N/2 is row 0, slot N/2 + j is row 1).
 */
#ifndef HE_H
#define HE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = -1,   /* bad argument: shape, size, domain, level or parameter */
    HE_ENOMEM = -2,   /* device allocation failed */
    HE_ENOKEY = -3,   /* a rotation needs a Galois key that is not loaded */
    HE_ECUDA = -4,    /* a CUDA call or kernel launch failed */
    HE_ETIMEOUT = -5  /* a bounded device-side wait ran out: reported by he_check and by the
                         synchronising calls that check the device error word (he_decrypt,
                         he_phase_times, he_ffconv_graph_create) */
};

enum { HE_COEFF = 0, HE_NTT = 1 };            /* representation of a ciphertext's limbs */
enum { HE_DP_DOT = 0, HE_DP_SHIFT = 1, HE_DP_SHIFT_EXT = 2, HE_CP_CP = 3, HE_DP_DP = 4 };  /* schedule */

/* Rotation step that swaps the two rows of slots (Galois element 2N - 1). */
#define HE_ROW_SWAP ((int32_t)0x7fffffff)
/* Pseudo-step naming the relinearisation key (switching s^2 back to s) in he_keygen_galois,
 * he_load_keys and he_export_galois; he_multiply needs it. */
#define HE_RELIN_KEY ((int32_t)0x80000000)

typedef struct he_ctx he_ctx;

/* BFV parameters (Sec. 2.1 fixes t, Q, N; the RNS split and key switching are readings).
 * The ciphertext primes q_0 > ... > q_{n_q-1} are the largest primes below 2^q_bits with
 * q = 1 mod 2N; the special primes p_0 > ... the largest below 2^p_bits with the same
 * congruence.  alpha primes form one key-switching digit (dnum = ceil(n_q / alpha)).
 * Limits: 6 <= log_n <= 16, 1 <= n_q <= 32, 1 <= n_p <= 8, 20 <= q_bits, p_bits <= 60,
 * 1 <= alpha <= n_q, alpha <= n_p (key-switching noise), t an odd prime < 2^62. */
typedef struct {
    uint32_t log_n;
    uint32_t n_q;
    uint32_t q_bits;
    uint32_t n_p;
    uint32_t p_bits;
    uint32_t alpha;
    uint64_t t;
} he_params;

/* A ciphertext in caller-owned device memory: data is [n_polys][n_limbs][N] uint64,
 * contiguous.  n_polys is 2; n_limbs is the level (n_q for fresh ciphertexts, one less
 * after he_rescale); domain is HE_COEFF or HE_NTT. */
typedef struct {
    uint64_t* data;
    uint32_t n_polys;
    uint32_t n_limbs;
    int32_t domain;
} he_ct;

/* Shape of one FFConv layer (Sec. 3.1 notation): input I_c x I_h x I_w, low-rank filters
 * W1 of d x d x I_c x r (r = O'_c of Eq. 2), restoring filters W2 of 1 x 1 x r x O_c,
 * stride and zero padding of W1, pack = HE_DP_DOT, HE_DP_SHIFT, HE_DP_SHIFT_EXT, HE_CP_CP or
 * HE_DP_DP (the DensePack-DensePack baseline of Table IX: W2 also under DensePack);
 * modswitch != 0 drops the last ciphertext prime at the end of the layer (not with HE_DP_DP). */
typedef struct {
    int32_t I_c, I_h, I_w, d, stride, pad, r, O_c;
    int32_t pack;
    int32_t modswitch;
} he_layout;

/* ---- context ---------------------------------------------------------------------- */

/* Create a context for `params` on the current CUDA device; `cuda_stream` is a
 * cudaStream_t (NULL = default stream).  Builds primes, twiddle and base-conversion
 * tables on the host and uploads them.  Errors: HE_EINVAL (parameters out of range or too
 * few primes), HE_ENOMEM, HE_ECUDA.  *out is NULL on error. */
int he_ctx_create(const he_params* params, void* cuda_stream, he_ctx** out);
void he_ctx_destroy(he_ctx* ctx);
/* Message of the last error on this context (never NULL; empty when none). */
const char* he_last_error(const he_ctx* ctx);
/* Change the stream later work is enqueued on. */
int he_set_stream(he_ctx* ctx, void* cuda_stream);
/* Copy the moduli to host memory: out[0..n_q) = q_i, out[n_q..n_q+n_p) = p_k, then t.
 * `cap` is the capacity of out; returns the count written or HE_EINVAL. */
int he_get_moduli(const he_ctx* ctx, uint64_t* out, int cap);
/* Operation counters since creation or the last reset: out[0] MulPC, out[1] AddCC,
 * out[2] rotations, out[3] key switches (Table I's counted operations). */
void he_op_counts(const he_ctx* ctx, uint64_t out[4]);
void he_reset_op_counts(he_ctx* ctx);
/* Number of CUDA kernels this context has launched since creation (a diagnostic). */
uint64_t he_launch_count(const he_ctx* ctx);
/* Phase timing (a diagnostic).  While enabled, he_ffconv_layer(_batch) brackets each phase
 * with CUDA events on the context stream: HE_PHASE_ENCODE (plaintexts from the weights),
 * HE_PHASE_MODUP (hoisting: inverse NTT of c1, ModUp, NTT of the digits), HE_PHASE_TAPS
 * (key switches and tap products: the fused extended-basis kernel, or the per-tap rotations
 * and MACs), HE_PHASE_MODDOWN (ModDown of the channel sums), HE_PHASE_ROTATE (DP_DOT
 * rotate-and-sum, channel folds and combines, fully connected rotate-and-sum),
 * HE_PHASE_RESTORE (W2 ConvPack and modulus switch), HE_PHASE_MULTIPLY (he_multiply(_batch):
 * lift, tensor, scale and relinearisation).  The fully connected layers time their diagonal
 * plaintexts, ModUp, tap sums and ModDown under the same phases as the FFConv layer.
 * he_phase_times synchronises the stream, writes the summed milliseconds of each phase to
 * ms_out[0..HE_N_PHASES) and the number of timed spans to calls_out (either may be NULL), and
 * clears the sums.  Enabling adds two event records per phase per call. */
enum { HE_PHASE_ENCODE = 0, HE_PHASE_MODUP = 1, HE_PHASE_TAPS = 2, HE_PHASE_MODDOWN = 3,
       HE_PHASE_ROTATE = 4, HE_PHASE_RESTORE = 5, HE_PHASE_MULTIPLY = 6, HE_N_PHASES = 8 };
int he_set_phase_timing(he_ctx* ctx, int enable);
int he_phase_times(he_ctx* ctx, double* ms_out, uint64_t* calls_out);
/* The 20 cumulative thresholds of the error sampler (sigma = 3.2, |e| <= 19), as
 * computed by the library: T[m] = floor(2^63 Pr(|e| <= m)), T[19] = 2^63. */
void he_gaussian_table(uint64_t out[20]);

/* ---- client side: keys, encryption, decryption (Sec. 1: the client holds the secret) */

/* Ternary secret key from `seed` (SplitMix64 stream 1): sk_out is host int64[N] in
 * {-1, 0, 1}.  Synchronous. */
int he_keygen_secret(he_ctx* ctx, uint64_t seed, int64_t* sk_out);
/* Generate Galois keys for the rotation `steps` (host int32[n_steps]; HE_ROW_SWAP allowed)
 * from the host secret `sk` (int64[N]) and `seed`, and keep them resident on the device.
 * Steps with the same Galois element share one key. */
int he_keygen_galois(he_ctx* ctx, const int64_t* sk, uint64_t seed, const int32_t* steps,
                     int n_steps);
/* Copy the resident key of `step` to host memory in the interchange layout
 * [dnum][2][n_q + n_p][N] uint64, coefficient domain, index 0 = b, 1 = a.  Synchronous.
 * HE_ENOKEY if absent. */
int he_export_galois(he_ctx* ctx, int32_t step, uint64_t* blob_out);
/* Load n_steps keys from the host blob (n_steps consecutive keys in the layout of
 * he_export_galois) and keep them resident; replaces a key with the same Galois element.
 * Every residue must lie below its modulus: otherwise (corrupted material) none of the keys
 * of this call is kept and HE_EINVAL is returned. */
int he_load_keys(he_ctx* ctx, const uint64_t* galois_blob, const int32_t* steps, int n_steps);
/* Encrypt the slot vector `slots` (host int64[N], taken mod t) under the host secret sk
 * with randomness from `seed` (streams 2 and 3).  out->data must hold [2][n_q][N]; the
 * result is in out->domain (HE_COEFF or HE_NTT, chosen by the caller). */
int he_encrypt(he_ctx* ctx, const int64_t* sk, const int64_t* slots, uint64_t seed, he_ct* out);
/* Decrypt `ct` (any level, either domain) under sk and decode: slots_out is host
 * int64[N] with values in [0, t).  Synchronous. */
int he_decrypt(he_ctx* ctx, const int64_t* sk, const he_ct* ct, int64_t* slots_out);

/* ---- server side: evaluation ---------------------------------------------------------- */

/* In-place change of representation (negacyclic NTT per limb, or its inverse). */
int he_to_ntt(he_ctx* ctx, he_ct* ct);
int he_to_coeff(he_ctx* ctx, he_ct* ct);
/* Encode slot values (host int64[N]) as a plaintext for he_mul_plain_acc: pt_out is device
 * [n_q][N], the centred lift of the encoding, NTT domain. */
int he_encode(he_ctx* ctx, const int64_t* slots, uint64_t* pt_out);
/* Rotation by `step` slots (Sec. 3.2, Fig. 1b): decrypt(out)[row][j] = decrypt(in)[row][j+step]
 * within each row of N/2 slots.  Automorphism X -> X^(5^step), then hybrid key switching.
 * in/out: NTT domain, same level, in may equal out.  HE_ENOKEY without the key. */
int he_rotate(he_ctx* ctx, const he_ct* in, int32_t step, he_ct* out);
/* he_rotate without any device allocation (the paper has no counterpart: this serves callers
 * that cannot allocate device memory when they rotate -- a process whose GPU memory is
 * already reserved by another allocator, or a request path that must not wait on
 * cudaMalloc/cudaFree).  Same arguments and the same ciphertext bits as he_rotate; its
 * key-switching scratch is one static device array of 16 MiB, held by every GPU that loads
 * the library until exit (enough for N = 2^13 with 3 + 1 primes or N = 2^14 with 6 + 2
 * primes; larger parameter sets are rejected with HE_EINVAL and a message giving the size
 * needed).  The first call on a device looks up the array's device address, so make it
 * before any stream capture.  All calls share the array: calls that overlap on the GPU race
 * on it and must be serialised by the caller.  Calls cudaMalloc/cudaFree never; refused
 * (HE_EINVAL) while a graph is being recorded, because recording would allocate the graph's
 * own pointer tables. */
int he_rotate_noalloc(he_ctx* ctx, const he_ct* in, int32_t step, he_ct* out);
/* The Galois automorphism X -> X^(5^step) (X -> X^(2N-1) for HE_ROW_SWAP) on both polynomials
 * of n ciphertexts, without key switching (the step the paper's rotation starts with, Sec.
 * 3.2): out[i] decrypts under s(X^g) to the rotated slots.  NTT domain, any level; out[i]
 * must not alias in[i].  Ciphertexts stored back to back (in and out alike) take one launch.
 * No key needed. */
int he_automorphism(he_ctx* ctx, const he_ct* in, int n, int32_t step, he_ct* out);
/* The same rotation applied to n ciphertexts in one batch (one key read per launch). */
int he_rotate_batch(he_ctx* ctx, const he_ct* in, int n, int32_t step, he_ct* out);
/* h rotations of one ciphertext sharing one ModUp of c1 (hoisting): outs[i] = rotation by
 * steps[i].  Its ciphertext bits differ from he_rotate's (the lift happens before the
 * automorphism); both decrypt identically. */
int he_rotate_hoisted(he_ctx* ctx, const he_ct* in, const int32_t* steps, int h, he_ct* outs);
/* The same for n ciphertexts rotated by the same h steps: outs[i h + s] = rotation of in[i] by
 * steps[s], each output bit-identical to he_rotate_hoisted's.  The ciphertexts go through the
 * key switch in batches (one ModUp per ciphertext, each step's key read once per batch).  No
 * output may alias an input (HE_EINVAL). */
int he_rotate_hoisted_batch(he_ctx* ctx, const he_ct* in, int n, const int32_t* steps, int h,
                            he_ct* outs);
/* MulPC + AddCC (Table I): acc += sum_i cts[i] * pts[i], pts device [n][level][N] NTT domain
 * (e.g. from he_encode).  acc and cts in the NTT domain, same level. */
int he_mul_plain_acc(he_ctx* ctx, const he_ct* cts, const uint64_t* pts, int n, he_ct* acc);
/* AddCC: out = a + b (same level and domain; out may alias an input). */
int he_add(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);
/* Ciphertext product with relinearisation (Sec. 2.1's homomorphic multiplication; with a = b
 * the square x^2 the paper uses as activation, Sec. 3): out decrypts to the slot-wise product.
 * Exactly round(t/Q (a0 + a1 s)(b0 + b1 s)) coefficient-wise -- the centred lifts are
 * multiplied over an auxiliary basis B (prod B > 16 N Q, chosen by the context), and every
 * rounding is decided exactly (128-bit fixed-point fractions, multi-word integers where those
 * cannot decide) -- then the s^2 component is key-switched with the key of step HE_RELIN_KEY.
 * a, b, out: NTT domain, full level (out may alias an input); at most 32 ciphertext primes.
 * HE_ENOKEY without the relinearisation key. */
int he_multiply(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);
/* The same for n pairs: out[i] = a[i] b[i] (out[i] may alias a[i] or b[i]); pairs with
 * a[i] == b[i] for every i take the square path (one lift instead of two). */
int he_multiply_batch(he_ctx* ctx, const he_ct* a, const he_ct* b, int n, he_ct* out);
/* Modulus switch: out = round(in / q_last), one limb fewer.  NTT domain in and out. */
int he_rescale(he_ctx* ctx, const he_ct* in, he_ct* out);

/* Encrypted FFConv layer, FFConv packing DP-HI2C-CP (Sec. 4.2, Fig. 4; Tables I-III).
 *   ct_in      one ciphertext (NTT domain, level n_q) holding the input image packed as the
 *              layout requires: HE_DP_DOT and HE_DP_DP slot ci*I_h*I_w + h*I_w + w;
 *              HE_DP_SHIFT(_EXT) slot ci*B_c + h*I_w + w with B_c = I_h*I_w for I_c = 1,
 *              else the next power of two.
 *   lowrank_w  host int32 [r][I_c][d][d] (W1), restore_w host int32 [O_c][r] (W2); weights
 *              are taken mod t.
 *   ct_out     O_c caller-owned ciphertexts (NTT domain; level n_q, or n_q - 1 with
 *              modswitch).  Output channel c holds y2[c, oh, ow] (mod t) at slot
 *              oh*O_w + ow (HE_DP_DOT) or (stride*oh)*I_w + stride*ow (the shift schedules).
 * HE_DP_DOT is the paper's DensePack: per output (c', o) a zero-padded filter product and
 * rotate-and-sum over ceil(log2(occupied slots)) steps (plus a row swap when the input fills
 * both rows), then one-hot masks move the r*S dot products into r ciphertexts.
 * HE_DP_SHIFT rotates the input once per filter tap (hoisted) and accumulates tap
 * plaintexts, then folds channels with rotations by B_c*2^k.  HE_DP_SHIFT_EXT uses the same
 * slots and plaintexts but keeps the hoisted rotations in the extended basis Q u P: the tap
 * products are summed there and divided by P once per low-rank channel (different ciphertext
 * bits from HE_DP_SHIFT, identical decryptions; at most 64 filter taps).  All finish with W2
 * under ConvPack (scalar products, no rotation).  Needs the Galois keys of the schedule.
 * HE_CP_CP is FFConv packing CP-HI2C-CP (Sec. 4.2 'ConvPack for W1', Fig. 5; the TinyNet
 * layer of Table VI): the client performs the Im2Col and ct_in holds K = d*d*I_c column
 * ciphertexts per image (image b's column k = (ci, i, j) at index b*K + k, holding the input
 * pixel under tap (i, j) of output o at slot o = oh*O_w + ow); W1 and W2 are both ConvPack
 * scalar products (MulPC r (K + O_c), Table II), no Galois key is needed, and output channel
 * c holds y2[c, oh, ow] at slot oh*O_w + ow.
 * HE_DP_DP is the DensePack-DensePack baseline of Table IX (LoLa's packing): W1 as HE_DP_DOT,
 * the r channel ciphertexts combined into one dense vector (channel c' rotated by -c'*S so
 * y1[c', o] sits at slot c'*S + o), then W2 under DensePack too: per output (c, o) the vector
 * times the plaintext holding W2[c][c'] at slot c'*S + o, rotate-and-sum with steps 1, 2, ..,
 * 2^(k2-1) where 2^k2 > (r-1)*S, and one-hot masks gather the O_c*S dot products (output slot
 * oh*O_w + ow, zero elsewhere).  Needs r*S <= N/2 and no modswitch; r - 1 + O_c*S*k2
 * rotations beyond HE_DP_DOT's. */
int he_ffconv_layer(he_ctx* ctx, const he_ct* ct_in, const int32_t* lowrank_w,
                    const int32_t* restore_w, const he_layout* layout, he_ct* ct_out);
/* The same layer on B independent ciphertexts with shared weights: ct_in[B],
 * ct_out[B * O_c] (image b's channel c at b * O_c + c).  Rotations of all B images by one
 * Galois element share each key read. */
int he_ffconv_layer_batch(he_ctx* ctx, const he_ct* ct_in, int B, const int32_t* lowrank_w,
                          const int32_t* restore_w, const he_layout* layout, he_ct* ct_out);
/* Layer plans: the weights of a layer kept on the device with its W1 plaintexts already
 * encoded (like the Galois keys, model state that a server holds across requests).
 * he_ffconv_plan copies the weights, encodes the plaintexts once (Montgomery form, Q u P for
 * HE_DP_SHIFT_EXT) and returns a plan id; he_ffconv_layer_planned then runs
 * he_ffconv_layer_batch without the encode step (same results); he_ffconv_plan_free releases it.
 * HE_EINVAL for an unknown plan. */
int he_ffconv_plan(he_ctx* ctx, const int32_t* lowrank_w, const int32_t* restore_w,
                   const he_layout* layout, int32_t* plan_out);
int he_ffconv_layer_planned(he_ctx* ctx, int32_t plan, const he_ct* ct_in, int B, he_ct* ct_out);
int he_ffconv_plan_free(he_ctx* ctx, int32_t plan);
/* Recorded call sequences (CUDA graphs).  he_graph_begin starts recording on this context:
 * the library calls that follow and only enqueue device work (rotations, products, layers,
 * networks: everything except the entry points below) run their host code but their kernels
 * and copies are recorded instead of executed, until he_graph_end returns the recording as a
 * graph id.  he_graph_launch replays a graph on the context stream with one submission; each
 * replay reads the device buffers the recorded calls read (whatever they hold then) and
 * writes the ones they wrote.  The caller keeps those buffers allocated while the graph lives.
 * Rules: the recorded calls must not need more scratch than the context holds, so run the
 * same calls once before recording (a call that would grow the scratch or the network buffer
 * fails with HE_EINVAL while recording); he_keygen_*, he_load_keys, he_export_galois,
 * he_encrypt, he_decrypt, he_encode, he_autotune, he_probe_int_mac, he_ffconv_plan(_free),
 * he_phase_times, he_set_stream, he_ffconv_graph_create, he_graph_launch and he_graph_free
 * refuse to run while recording (HE_EINVAL).
 * Scratch: share_scratch = 1 records on the context's scratch (no extra memory; safe because
 * all of a context's work runs in order on its stream), valid until a later call reallocates
 * it; 0 gives the graph a scratch area of its own (of the context's current size).  The
 * resident keys, layer plans and network buffer are used by reference: new key material for
 * the same steps is picked up, while a launch after a used plan was freed, a key was dropped,
 * or the shared scratch or network buffer was reallocated fails with HE_EINVAL (record
 * again).  If any call fails while recording (refused ones included), he_graph_end discards
 * the recording and returns that call's error code.  he_graph_free releases a graph (after
 * the stream drains). */
int he_graph_begin(he_ctx* ctx, int share_scratch);
int he_graph_end(he_ctx* ctx, int32_t* graph_out);
/* A planned layer recorded in one call: he_ffconv_layer_planned(plan, ct_in, B, ct_out) runs
 * once (ct_out holds its result on return; for share_scratch = 0 it sizes a scratch area the
 * graph keeps), then is recorded on these exact buffers. */
int he_ffconv_graph_create(he_ctx* ctx, int32_t plan, const he_ct* ct_in, int B, he_ct* ct_out,
                           int share_scratch, int32_t* graph_out);
int he_graph_launch(he_ctx* ctx, int32_t graph);
int he_graph_free(he_ctx* ctx, int32_t graph);
/* Rotation steps the layer needs keys for; writes at most `cap` steps into steps_out and
 * returns the count (or HE_EINVAL for a layout that does not fit the ring). */
int he_ffconv_required_steps(const he_ctx* ctx, const he_layout* layout, int32_t* steps_out,
                             int cap);

/* ---- three-layer network (Table VIII's pipeline) ---------------------------------- */

/* Fully connected layer as DensePack dot products (Sec. 3: a fully connected layer is a
 * convolution whose filter covers the whole input), on B ciphertexts with shared weights.
 * Input value x_i sits at slot pos[i] of row 0 and repeats with period `period` (a power of
 * two, M <= period <= N/2 with M the smallest power of two >= n_out; period = N/2 for an
 * input that does not repeat; row 1 and every other slot of a period must be zero).
 * weights: host int32 [n_out][n_in]; pos: host int32 [n_in], distinct, in [0, period).
 * Output: y_j = sum_i weights[j][i] x_i (mod t) at every slot p of row 0 with p mod M = j,
 * zero where p mod M >= n_out (the output repeats with period M).  Schedule: the M diagonal
 * plaintexts diag_k[p] = weights[p mod M][i] where (p + k) mod period = pos[i]; the M - 1
 * hoisted rotations of x summed with them in Q u P and divided by P once; then
 * log2(period / M) rotate-and-sum steps z <- z + rot(z, M 2^e).  Keys: steps 1 .. M-1 and
 * M 2^e.  in, out: full level, NTT domain (out may alias in). */
int he_fc_layer_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* weights,
                      const int32_t* pos, int n_in, int n_out, int period, he_ct* out);
/* Channel combine (Table VIII, "combine to one vector"): out[b] = in[b n_ch] +
 * sum_{c >= 1} rot(in[b n_ch + c], -c block), n_ch - 1 rotations per image.  in: [B][n_ch]
 * ciphertexts, full level, NTT domain. */
int he_combine_batch(he_ctx* ctx, const he_ct* in, int B, int n_ch, int block, he_ct* out);

/* Shape of the network: the FFConv layer (modswitch 0, outputs in row 0), then x^2, a fully
 * connected layer of m1 outputs over the O_c O_h O_w layer outputs (flattened in
 * (c, oh, ow) order), x^2, and a fully connected layer of m2 outputs. */
typedef struct {
    he_layout conv;
    int32_t m1, m2;
} he_net;
/* Steps whose keys the network needs (the layer's, the combine's -c blk mod N/2, both
 * fully connected layers'), then HE_RELIN_KEY; count returned, at most cap written. */
int he_net_required_steps(const he_ctx* ctx, const he_net* net, int32_t* steps_out, int cap);
/* The network on B images: he_ffconv_layer_batch, he_combine_batch with block = the smallest
 * power of two above every layer output slot, he_multiply_batch (square), he_fc_layer_batch
 * (positions c block + slot(oh, ow), period N/2), square, he_fc_layer_batch (positions
 * 0 .. m1-1, period next_pow2(m1)).  in: B ciphertexts (B K Im2Col columns for HE_CP_CP);
 * lowrank_w / restore_w as for the layer; fc1_w host int32 [m1][O_c O_h O_w]; fc2_w host
 * int32 [m2][m1]; out[B]: full level, z2_j at slots p of row 0 with p mod next_pow2(m2) = j.
 * Intermediate ciphertexts live in a context-owned device buffer (grow-only). */
int he_net_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* lowrank_w,
                 const int32_t* restore_w, const int32_t* fc1_w, const int32_t* fc2_w,
                 const he_net* net, he_ct* out);

/* ---- deeper networks over several ciphertexts per tensor --------------------------- */

/* A stride-1 "same" convolution layer (d odd, pad = (d - 1) / 2) on a C_in x H x W tensor:
 * factorized (Eq. 2) into r low-rank d x d filters and a 1 x 1 restore to O_c channels, or
 * unfactorized (r = 0: O_c d x d filters, no restore). */
typedef struct {
    int32_t C_in, H, W, d, pad, r, O_c;
} he_mc_conv;
/* Tensor layout of these calls: channel c of the H x W map occupies block c mod g of ciphertext
 * c / g (row 0), block size Bk = next_pow2(H W), g = (N/2) / Bk, pixel (h, w) at offset
 * h W + w; other slots zero.  Packing (DensePack over several ciphertexts, Sec. 3.2 with the
 * FFConv factorization of Sec. 4): every input ciphertext is rotated by the d^2 - 1 nonzero tap
 * offsets (hoisted, summed in Q u P per low-rank channel over all input ciphertexts, one
 * ModDown each); the block sum y1 = sum_{u<g} rot(acc, u Bk) (g - 1 rotations hoisted from one
 * ModUp, summed in Q u P, one ModDown) replicates each low-rank output in every block; output
 * ciphertext G = sum_c' y1[c'] * P[G][c'] with P[G][c'] holding
 * restore_w[G g + j][c'] on block j (identity when unfactorized) -- no rotation.  in:
 * [B][ceil(C_in / g)], out: [B][ceil(O_c / g)], full level, NTT domain.  lowrank_w: host int32
 * [r or O_c][C_in][d][d]; restore_w: host int32 [O_c][r], NULL when r = 0.  Keys: the nonzero
 * tap offsets (i - pad) W + (j - pad) and the block steps u Bk, u = 1 .. g - 1. */
int he_mc_conv_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* lowrank_w,
                     const int32_t* restore_w, const he_mc_conv* conv, he_ct* out);
/* In place, for each step in order: x <- x + rot(x, step), on n ciphertexts (full level, NTT
 * domain); e.g. a sum pooling inside blocks of Bk slots (steps 1, 2, ..., Bk/2). */
int he_rotate_sum_batch(he_ctx* ctx, he_ct* cts, int n, const int32_t* steps, int n_steps);
/* he_fc_layer_batch over n_ct input ciphertexts per image (in: [B][n_ct]): feature i at slot
 * pos[i] of ciphertext ct_of[i]; the taps of all input ciphertexts are summed in Q u P before the
 * one ModDown.  Keys as for he_fc_layer_batch. */
int he_fc_mc_batch(he_ctx* ctx, const he_ct* in, int B, int n_ct, const int32_t* weights,
                   const int32_t* ct_of, const int32_t* pos, int n_feat, int n_out, int period,
                   he_ct* out);
/* Steps whose keys he_deep_batch needs (layer taps and folds, classifier), then HE_RELIN_KEY;
 * count returned, at most cap written. */
int he_deep_required_steps(const he_ctx* ctx, const he_mc_conv* convs, int n_layers, int n_cls,
                           int32_t* steps_out, int cap);
/* The deeper network on B images: for each layer he_mc_conv_batch then the square
 * (he_multiply_batch) of every output ciphertext; then global sum pooling and a fully
 * connected layer to n_cls classes, evaluated together as one fully connected layer over every
 * activation (feature (c, pixel) weighted fc_w[j][c]; he_fc_mc_batch, period N/2) -- the
 * pooling costs no rotation.  lowrank_w[l] / restore_w[l] as for he_mc_conv_batch
 * (restore_w[l] NULL for unfactorized layers); fc_w host int32 [n_cls][O_c of the last layer].
 * in: [B][ceil(C0 / g)] packed as above; out[B]: class j at slots p of row 0 with
 * p mod next_pow2(n_cls) = j.  Intermediate ciphertexts live in a context-owned buffer. */
int he_deep_batch(he_ctx* ctx, const he_ct* in, int B, const he_mc_conv* convs, int n_layers,
                  const int32_t* const* lowrank_w, const int32_t* const* restore_w,
                  const int32_t* fc_w, int n_cls, he_ct* out);

/* ---- tuning ------------------------------------------------------------------------ */

/* Autotuner of implementation parameters (no counterpart in the paper; results never depend
 * on them): (1) the split N = N1 N2 of the two-pass NTT and its radix (rounds of up to 8 or
 * up to 4 points per thread group), timing forward + inverse transforms of `batch`
 * ciphertexts for each candidate pair; (1b) the limb groups of the ModUp / ModDown base
 * conversions (a thread converts all target limbs of a digit, half of them or a quarter: 1,
 * 2 or 4 groups across the grid), timed on `batch` ciphertexts; (2) the fused tap kernel's
 * tile (128 or 256
 * coefficients per CTA) and its arithmetic -- 0: 64 x 64-bit products in 32-bit multiply-add
 * carry chains; 1: 30-bit halves summed into 64-bit columns; 2: the plaintext x key products
 * precomputed per launch and every tap summed unreduced in 25-bit-split columns (ciphertext
 * primes below 2^50 only; the special-prime limbs then take the carry chains) -- timing each
 * on synthetic operands of `batch` images (25 taps, 2 channels, this context's key shape).
 * The fastest of each is kept for every later call on the context.  force_tile = 128 or 256
 * only sets the tile, without timing.  ms_out (HE_TUNE_REPORT_LEN doubles, may be NULL):
 * [0..3] tap-kernel ms per launch for (tile 128, chains), (128, columns), (256, chains),
 * (256, columns); [4] the NTT time of the chosen split and [5] its log2 N1; [6] the chosen
 * tile; [7] the chosen arithmetic; [8] the precomputed-product path's ms (0 where it does not
 * apply); [9] the chosen NTT radix (8 or 4); [10..12] the conversions' ms with 1, 2 and 4
 * limb groups and [13] the chosen number; [14] / [15] one ModUp + ModDown of min(batch, 64)
 * ciphertexts with the base conversions as separate kernels / inside the forward NTT's first
 * pass (the faster is kept, HE_TUNE_BCONV_FUSED).  Without a call: tile 128 for keys of four or more digits (else 256),
 * carry chains, split log2 N1 = floor(log2 N / 2).  Uses the context scratch; synchronises
 * the stream. */
#define HE_TUNE_REPORT_LEN 16
int he_autotune(he_ctx* ctx, int batch, int force_tile, double* ms_out);
/* Tuning knobs, set by hand (value -1 restores the default) or read back: HE_TUNE_TAP_TILE
 * (128 or 256), HE_TUNE_TAP_ARITH (0 chains, 1 columns, 2 precomputed products),
 * HE_TUNE_NTT_SPLIT (log2 N1, 1 .. log2 N - 1), HE_TUNE_NTT_RADIX (4 or 8: the most points
 * a thread group transforms per round), HE_TUNE_LIMB_GROUPS (1, 2 or 4), HE_TUNE_BCONV_FUSED
 * (0: the ModUp / ModDown base conversions as separate kernels, 1 (default): read by the
 * forward NTT's first pass, the inverse NTT before them leaving y directly).  Results never
 * depend on them.  he_tune_set is
 * refused while recording.  The precomputed products take a grow-only buffer of 16 x taps x
 * dnum x n_q x N bytes, allocated at the first call that needs it (not while recording). */
enum {
    HE_TUNE_TAP_TILE = 0,
    HE_TUNE_TAP_ARITH = 1,
    HE_TUNE_NTT_SPLIT = 2,
    HE_TUNE_NTT_RADIX = 3,
    HE_TUNE_LIMB_GROUPS = 4,
    HE_TUNE_BCONV_FUSED = 5
};
int he_tune_set(he_ctx* ctx, int knob, int value);
int he_tune_get(he_ctx* ctx, int knob, int* value);

/* ---- failure detection ------------------------------------------------------------ */

/* Waits for the context's stream, then reports HE_ECUDA if a kernel failed, HE_ETIMEOUT if a
 * bounded device-side wait of a kernel enqueued since the last check ran out (the results of
 * that work are unusable; the error word is cleared, so the next check starts afresh), else
 * HE_OK.  The only device-side waits are the fused tap kernel's waits on its shared-memory
 * stages (he_ffconv_layer with HE_DP_SHIFT_EXT and the network and multi-ciphertext calls
 * built on it).  Refused while recording.  Synchronous. */
int he_check(he_ctx* ctx);
/* Test hook for the path above (no counterpart in the paper): the fused tap kernel's compute
 * warps report their wait for a stage's operands (error bit set) once it has polled `polls`
 * times, then keep waiting up to the full bound (2^20 polls), so copies and results stay in
 * step and only the report is forced.  polls = 0 reports every such wait; polls < 0 restores
 * the default (reports only at the full bound).  Refused while recording. */
int he_set_wait_report(he_ctx* ctx, int polls);

/* ---- primitives for measurement --------------------------------------------------- */

/* Microbenchmark of the 64 x 64 -> 128-bit multiply-accumulate rate (registers only, eight
 * independent accumulators per thread, 8 CTAs of 256 threads per SM): out[0] = products/s of
 * the 32-bit multiply-add carry chain the kernels use, out[1] = products/s with 30-bit limbs
 * summed into 64-bit column accumulators.  Uses the context stream and scratch; synchronous. */
int he_probe_int_mac(he_ctx* ctx, double* out);
/* The same probe per form and per instruction (n doubles, up to 6): out[0] carry-chain
 * products/s, out[1] column products/s, out[2] products/s with three 32 x 32 -> 64-bit
 * products each (Karatsuba on 30-bit halves), out[3] mad.lo.u32/s, out[4] mad.hi.u32/s,
 * out[5] mad.wide.u32/s (eight independent accumulators per thread), out[6] products/s of the
 * 64-bit add-with-carry form for operands below 2^63 (the kernels' residue products).
 * Synchronous. */
int he_probe_int_ops(he_ctx* ctx, double* out, int n);
/* Read bandwidth in GB/s (n doubles, up to 2): out[0] of a 32 MiB buffer that stays in L2,
 * out[1] of a 2 GiB buffer read from HBM (16-byte loads bypassing L1, all SMs).  Uses the
 * context stream and scratch; synchronous. */
int he_probe_mem(he_ctx* ctx, double* out, int n);

/* Negacyclic NTT (inverse = 0) or inverse NTT (inverse = 1) in place on `n_items` blocks of
 * n_limbs limbs each (device [n_items][n_limbs][N]); limb i uses the i-th ciphertext prime
 * (i < n_q) or the (i - n_q)-th special prime. */
int he_ntt(he_ctx* ctx, uint64_t* data, int n_items, int n_limbs, int inverse);

#ifdef __cplusplus
}
#endif

#endif /* HE_H */
