// he_internal.cuh -- shared declarations of the GB300 RNS-BFV library (not part of the ABI).
//
// Modular arithmetic on 64-bit residues (moduli below 2^62), built from the 64-bit integer
// multiply of the SM (lowered to 32-bit IMAD):
//   * Shoup products x*w mod q for a constant w with companion w' = floor(w 2^64 / q):
//     r = x w - floor(x w' / 2^64) q lies in [0, 2q) for any 64-bit x;
//   * Montgomery reduction REDC(x) = x 2^-64 mod q for a 128-bit x < q 2^64, used to reduce
//     sums of products once (key-switch inner products, plaintext MACs); constants stored in
//     Montgomery form (w 2^64 mod q) make REDC return plain residues.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "he.h"

#define HE_MAX_MODS 48

struct ModConst {
    uint64_t q;
    uint64_t qinv_neg;   // -q^-1 mod 2^64
    uint64_t r2;         // 2^128 mod q (to Montgomery form via REDC(x r2))
    uint64_t n_inv;      // N^-1 mod q
    uint64_t n_inv_sh;   // its Shoup companion
    uint64_t one_sh;     // floor(2^64 / q): Shoup companion of 1 (x mod q for any 64-bit x)
    // quotient estimate for values below 2^(b + 7), b = bit length of q <= 57 (reduce_small):
    // red_r = floor(2^(31 + b) / q), red_sh = max(b - 25, 0), red_t = 31 + b - red_sh
    uint32_t red_r;
    uint16_t red_sh, red_t;
};

struct ShoupPair {
    uint64_t w, ws;
};

// ------------------------------------------------------------------ device arithmetic

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

// v mod q for v < 2^(b + 7) (b = bit length of q, at most 57).  With vh = floor(v / 2^sh)
// (below 2^32) the estimate k = floor(vh red_r / 2^t) satisfies floor(v/q) - 1 <= k <=
// floor(v/q): each truncation costs less than 2^-24 of a quotient unit.  So v - k q lies in
// [0, 2q) and one conditional subtraction finishes.
__device__ __forceinline__ uint64_t reduce_small(uint64_t v, const ModConst& M) {
    const uint32_t vh = (uint32_t)(v >> M.red_sh);
    const uint32_t k = (uint32_t)(((uint64_t)vh * M.red_r) >> M.red_t);
    const uint64_t r = v - (uint64_t)k * M.q;
    return r >= M.q ? r - M.q : r;
}

__device__ __forceinline__ uint64_t neg_mod(uint64_t a, uint64_t q) { return a ? q - a : 0; }

__device__ __forceinline__ uint32_t brv_bits(uint32_t x, int bits) {
    return bits ? (__brev(x) >> (32 - bits)) : 0u;
}

// NTT-domain automorphism X -> X^g: position p holds a(psi^(2 brv(p) + 1)); the image takes
// the value at exponent (2 brv(p) + 1) g mod 2N.
__device__ __forceinline__ uint32_t perm_src(uint32_t p, uint32_t g, int logN) {
    uint32_t e = (2u * brv_bits(p, logN) + 1u) * g & ((2u << logN) - 1u);
    return brv_bits((e - 1u) >> 1, logN);
}

// High 64 bits of a 64 x 64-bit product from 32-bit partial products in one carry chain (the
// low word of a0 b0 cannot carry: it is never added to).
#pragma nv_diag_suppress 550   // c1 below is written by the chain and read only through carries
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t c1, c2, c3;
    asm("mul.hi.u32 %0, %3, %5;\n\t"
        "mul.lo.u32 %1, %4, %6;\n\t"
        "mul.hi.u32 %2, %4, %6;\n\t"
        "mad.lo.cc.u32 %0, %3, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %6, %1;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        "mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %5, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=&r"(c1), "=&r"(c2), "=&r"(c3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    return ((uint64_t)c3 << 32) | c2;   // c1 (bits 32..63) only feeds the carries
}
#pragma nv_diag_default 550

// x * w mod q, x any 64-bit value, w < q, ws = floor(w 2^64 / q).
__device__ __forceinline__ uint64_t mul_shoup(uint64_t x, uint64_t w, uint64_t ws, uint64_t q) {
    uint64_t h = mulhi64(x, ws);
    uint64_t r = x * w - h * q;
    return r >= q ? r - q : r;
}

// Same, result left in [0, 2q).
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t x, uint64_t w, uint64_t ws,
                                                   uint64_t q) {
    uint64_t h = mulhi64(x, ws);
    return x * w - h * q;
}

// Same with the high product estimated from three of the four partial products:
// h' = x1 w1 + hi(x0 w1) + hi(x1 w0) is floor(x ws / 2^64) minus 0, 1 or 2 (the dropped low
// halves and hi(x0 w0) carry at most 2 into bit 64), so x w - h' q lies in [0, 4q).
__device__ __forceinline__ uint64_t mul_shoup_approx(uint64_t x, uint64_t w, uint64_t ws,
                                                     uint64_t q) {
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t w0 = (uint32_t)ws, w1 = (uint32_t)(ws >> 32);
    uint64_t h = (uint64_t)__umulhi(x0, w1) + __umulhi(x1, w0);
    h += (uint64_t)x1 * w1;
    return x * w - h * q;
}

struct U128 {
    uint64_t lo, hi;
};

// acc += a * b (128-bit accumulator, 64 x 64-bit product): the four 32 x 32-bit partial
// products are added in one carry chain of 32-bit multiply-adds (ten instructions), on the
// 32-bit halves of 64-bit operands split inside the block.
__device__ __forceinline__ void mac128(U128& acc, uint64_t a, uint64_t b) {
    asm("{\n\t.reg .u32 a0, a1, b0, b1, c0, c1, c2, c3;\n\t"
        "mov.b64 {a0, a1}, %2;\n\t"
        "mov.b64 {b0, b1}, %3;\n\t"
        "mov.b64 {c0, c1}, %0;\n\t"
        "mov.b64 {c2, c3}, %1;\n\t"
        "mad.lo.cc.u32 c0, a0, b0, c0;\n\t"
        "madc.hi.cc.u32 c1, a0, b0, c1;\n\t"
        "madc.lo.cc.u32 c2, a1, b1, c2;\n\t"
        "madc.hi.u32 c3, a1, b1, c3;\n\t"
        "mad.lo.cc.u32 c1, a0, b1, c1;\n\t"
        "madc.hi.cc.u32 c2, a0, b1, c2;\n\t"
        "addc.u32 c3, c3, 0;\n\t"
        "mad.lo.cc.u32 c1, a1, b0, c1;\n\t"
        "madc.hi.cc.u32 c2, a1, b0, c2;\n\t"
        "addc.u32 c3, c3, 0;\n\t"
        "mov.b64 %0, {c0, c1};\n\t"
        "mov.b64 %1, {c2, c3};\n\t}"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// acc += a * b for operands below 2^63 (residues): then the two cross products a0 b1 + a1 b0
// fit one 64-bit word, and the partial products enter the 128-bit sum by 64-bit add-with-carry
// (four 32 x 32 -> 64-bit multiplies, two shifts, four adds).  Measured 11 % more products per
// clock than mac128's 32-bit carry chain (5.94 against 5.36 per SM and clock on GB300).
__device__ __forceinline__ void mac128r(U128& acc, uint64_t a, uint64_t b) {
    asm("{\n\t.reg .u32 a0, a1, b0, b1;\n\t.reg .u64 lo, hi, mid, sh;\n\t"
        "mov.b64 {a0, a1}, %2;\n\t"
        "mov.b64 {b0, b1}, %3;\n\t"
        "mul.wide.u32 lo, a0, b0;\n\t"
        "mul.wide.u32 hi, a1, b1;\n\t"
        "mul.wide.u32 mid, a0, b1;\n\t"
        "mad.wide.u32 mid, a1, b0, mid;\n\t"
        "add.cc.u64 %0, %0, lo;\n\t"
        "addc.u64 %1, %1, hi;\n\t"
        "shl.b64 sh, mid, 32;\n\t"
        "shr.u64 mid, mid, 32;\n\t"
        "add.cc.u64 %0, %0, sh;\n\t"
        "addc.u64 %1, %1, mid;\n\t}"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// REDC: x 2^-64 mod q for x < q 2^64, result in [0, q).  With m = x q' mod 2^64 the sum
// x + m q is divisible by 2^64 and its top half is x 2^-64 mod q, in [0, 2q).
__device__ __forceinline__ uint64_t redc(U128 x, uint64_t q, uint64_t qinv_neg) {
    const uint64_t m = x.lo * qinv_neg;
    mac128(x, m, q);
    const uint64_t t = x.hi;
    return t >= q ? t - q : t;
}

__device__ __forceinline__ uint64_t to_mont(uint64_t a, const ModConst& M) {
    U128 x{0, 0};
    mac128(x, a, M.r2);
    return redc(x, M.q, M.qinv_neg);
}

// ------------------------------------------------------------------ host-side context

struct Arena {
    // Grow-only device scratch.  take() hands out 256-byte aligned slices of one buffer;
    // reset() frees every slice at once.  Growing synchronises the stream first.
    char* base = nullptr;
    size_t cap = 0, used = 0;
};

struct Staging {
    // Pinned host slots + device slots for small uploads (pointer tables, weights).
    static constexpr int kSlots = 64;
    size_t slot_bytes = 1 << 18;
    int n_slots = kSlots;
    int next = 0;
    char* host = nullptr;
    char* dev = nullptr;
    cudaEvent_t ev[kSlots] = {};
};

struct GaloisKey {
    uint64_t* dev = nullptr;     // [dnum][2][L+K][N], NTT domain, Montgomery form
};

struct he_ctx {
    he_params prm{};
    int N = 0, logN = 0, L = 0, K = 0, alpha = 0, dnum = 0;
    int n_mod = 0;               // L + K + 1 + n_b: q's, p's, t, then the auxiliary basis B
    int n_b = 0;                 // auxiliary primes for ciphertext multiplication (prod B > N Q)
    uint64_t* d_mult_tab = nullptr;   // exact extension + scale-and-round tables (mult.cu)
    size_t mult_ext_words = 0, mult_extf_off = 0, mult_scf_off = 0;
    int mult_Wq = 0, mult_Wm = 0;
    bool batching = false;       // t = 1 mod 2N: slot encoding available
    std::vector<uint64_t> mods;  // q_0..q_{L-1}, p_0..p_{K-1}, t
    cudaStream_t stream = nullptr;

    ModConst* d_mod = nullptr;          // [n_mod]
    ShoupPair* d_tw_fwd = nullptr;      // [n_mod][N]: psi^brv(k)
    ShoupPair* d_tw_inv = nullptr;      // [n_mod][N]: psi^-brv(k)
    // d_tw_fwd with each forward row-pass stage reordered so that a round's lanes read
    // consecutive entries (ntt.cu ensure_row_tables); valid for the split and radix cap here
    ShoupPair* d_tw_fwd_rows = nullptr;
    int tw_rows_s1 = -1, tw_rows_k = -1;
    int32_t* d_slot_pos = nullptr;      // [N]: NTT position of each slot (mod t, root zeta)
    uint64_t* d_cdt = nullptr;          // [20] sampler thresholds
    // ModUp: y_i = x_i [(Q_j/q_i)^-1]_{q_i};  then sum_i y_i [Q_j/q_i]_{p_l}
    ShoupPair* d_modup_inv = nullptr;   // [L]
    ShoupPair* d_modup_c = nullptr;     // [dnum][alpha][L+K]
    // ModDown: y_k = u_k [(P/p_k)^-1]_{p_k}; v_i = sum_k y_k [P/p_k]_{q_i}; (u_i - v_i) P^-1
    ShoupPair* d_md_inv = nullptr;      // [K]
    ShoupPair* d_md_c = nullptr;        // [K][L]
    ShoupPair* d_md_pinv = nullptr;     // [L]
    // the inverse NTT's N^-1 times the conversion's first factor, so that the inverse transform
    // of a converted limb leaves y directly (the fused conversion, ntt_forward_bconv)
    ShoupPair* d_modup_ninv = nullptr;  // [L]: N^-1 [(Q_j/q_i)^-1]_{q_i}
    ShoupPair* d_md_ninv = nullptr;     // [K]: N^-1 [(P/p_k)^-1]_{p_k}
    ShoupPair* d_rs_inv = nullptr;      // [L][L]: row lv = q_lv^-1 mod q_i (rescale at level lv+1)
    uint64_t* d_pmodq = nullptr;        // [L] P mod q_i (Montgomery form) for key generation
    int* d_err = nullptr;               // device error word: bit 0 = a bounded wait ran out

    std::map<uint32_t, GaloisKey> keys; // by Galois element
    Arena arena;
    Arena net;                          // ciphertexts between the layers of he_net_batch
    Arena pk;                           // the tap kernel's plaintext x key products (tapmac.cu)
    int tap_tile = 0;                   // tap kernel tile chosen by he_autotune (0: default)
    int ntt_s1 = 0;                     // NTT split log2 N1 chosen by he_autotune (0: default)
    int ntt_radix = 0;                  // NTT rounds of up to 2^ntt_radix points (0: 3, radix 8)
    int limb_groups = 0;                // ModUp / ModDown conversions: target limbs split in
                                        // this many groups across the grid (0: 1)
    int bconv_fused = 1;                // ModUp / ModDown base conversions: 1 inside the
                                        // forward NTT's first pass, 0 separate kernels
    int tap_arith = 0;                  // tap kernel: 0 carry chains, 1 30-bit columns,
                                        // 2 precomputed plaintext x key products
    int wait_report = -1;               // he_set_wait_report: polls before a stage wait is
                                        // reported in the tap kernel (-1: the full bound)
    struct LayerPlan {                  // he_ffconv_plan: weights and encoded W1 plaintexts
        he_layout layout;
        std::vector<int32_t> w1, w2;
        uint64_t* pts = nullptr;        // device, NULL for HE_CP_CP
    };
    std::map<int32_t, LayerPlan> plans;
    int32_t next_plan = 1;
    uint64_t keys_epoch = 0;            // bumped whenever a resident key is dropped
    uint64_t arena_epoch = 0;           // bumped whenever the scratch arena is reallocated
    uint64_t net_epoch = 0;             // bumped whenever the network buffer is reallocated
    uint64_t pk_epoch = 0;              // bumped whenever the tap products buffer is reallocated
    struct LayerGraph {                 // a recorded sequence of library calls (graph.cu)
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        Arena arena;                    // the graph's own scratch (empty when shared)
        bool shared = false;            // recorded on the context's scratch
        uint64_t arena_epoch = 0;       // ... at this generation of it
        uint64_t net_epoch = 0;         // network buffer generation at recording
        uint64_t pk_epoch = 0;          // tap products buffer generation at recording
        uint64_t keys_epoch = 0;
        std::vector<void*> allocs;      // small tables uploaded while recording
        std::vector<int32_t> plans;     // layer plans the recorded calls use
        uint64_t launches = 0, ops[4] = {0, 0, 0, 0};   // per replay
    };
    std::map<int32_t, LayerGraph> graphs;
    int32_t next_graph = 1;
    // While recording (he_graph_begin .. he_graph_end): the graph being built, the user's
    // stream and scratch to restore, and the counters to roll back.  Small uploads then go to
    // device buffers the graph owns instead of the reused staging ring, and the scratch and
    // network buffers refuse to grow.
    struct Recording {
        LayerGraph g;
        cudaStream_t user_stream = nullptr, cs = nullptr;
        Arena saved;
        bool timing = false;
        int failed = 0;                 // first error code of a call made while recording
        uint64_t launches0 = 0, ops0[4] = {0, 0, 0, 0};
    };
    Recording* rec = nullptr;
    Staging staging;
    uint64_t ops[4] = {0, 0, 0, 0};     // MulPC, AddCC, Rot, KeySwitch
    uint64_t launches = 0;              // kernels launched by this context
    // NVTX range of the phase in progress (shown by profilers that record NVTX; a no-op
    // otherwise)
    uint64_t nvtx_id = 0;
    bool nvtx_open = false;
    // optional per-phase timing (CUDA events on the context stream, summed on request)
    bool timing = false;
    struct PhaseSpan {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<PhaseSpan> spans;
    std::vector<cudaEvent_t> event_pool;
    double phase_ms[HE_N_PHASES] = {};
    uint64_t phase_calls[HE_N_PHASES] = {};
    std::string err;
};

// ------------------------------------------------------------------ internal helpers

#define HE_CHECK_CUDA(ctx, call)                                                       \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) return he_fail((ctx), HE_ECUDA, cudaGetErrorString(_e)); \
    } while (0)

int he_fail(he_ctx* ctx, int code, const std::string& msg);
// Entry points that synchronise, return host data or change resident state refuse to run
// while a graph is being recorded.
#define HE_NOT_RECORDING(ctx, name)                                                    \
    do {                                                                               \
        if ((ctx)->rec) return he_fail((ctx), HE_EINVAL, name ": not while recording a graph"); \
    } while (0)
// Ends and discards a recording in progress (context teardown).
void recording_abort(he_ctx* ctx);
// Synchronise the stream and report HE_ETIMEOUT if a kernel's bounded wait ran out.
int check_device_error(he_ctx* ctx);
int he_launch_check(he_ctx* ctx, const char* what);

uint64_t* arena_take(he_ctx* ctx, size_t n_u64);
void arena_reset(he_ctx* ctx);
int arena_reserve(he_ctx* ctx, size_t n_u64);
// The context's buffer for a network's activations (grow-only, like the arena).
int net_reserve(he_ctx* ctx, size_t n_u64);
// The tap kernel's buffer of plaintext x key products (grow-only, like the arena).
int pk_reserve(he_ctx* ctx, size_t n_u64);

uint32_t galois_elt(const he_ctx* ctx, int32_t step);
// Phase timing: phase_begin/phase_end bracket work of one phase (HE_PHASE_*) with events on
// the context stream when timing is enabled; no-ops otherwise.
void phase_begin(he_ctx* ctx, int phase);
void phase_end(he_ctx* ctx);
const void* upload_small(he_ctx* ctx, const void* src, size_t bytes);
int upload_host(he_ctx* ctx, void* dst, const void* src, size_t bytes);
const void* upload_args(he_ctx* ctx, const void* src, size_t bytes, void* scratch);
int check_ct(he_ctx* ctx, const he_ct* ct, int need_limbs, int need_domain, const char* what);
// Slot values (items x N int64, device) -> plaintexts [items][rows][N]: centred lift modulo
// the first `rows` moduli (L for Q, L + K for Q u P), NTT domain, Montgomery form if mont.
void encode_device(he_ctx* ctx, const int64_t* d_slots, int items, uint64_t* tmp, uint64_t* out,
                   int mont, int rows);
int he_get_key(he_ctx* ctx, uint32_t g, const uint64_t** key);
// Frees a captured layer's graph, scratch and tables (graph.cu); the stream must be idle.
void graph_release(he_ctx::LayerGraph& g);

// host arithmetic (api.cu)
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t q);
uint64_t h_inv(uint64_t a, uint64_t q);
ShoupPair h_shoup(uint64_t w, uint64_t q);
uint64_t h_to_mont(uint64_t x, uint64_t q);
uint64_t he_stream_state(uint64_t seed, uint64_t stream);
void he_cdt_compute(uint64_t out[20]);

// NTT launchers (ntt.cu).  A launch covers `items` blocks (stride `item_stride` u64) of
// `rows` consecutive limbs; limb r of a block uses modulus index mod_off + r.
void ntt_forward(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off);
// Brings the row-pass twiddle tables to the context's split and radix cap; called wherever
// those change (never while recording).
void ntt_prepare(he_ctx* ctx);
// Splits log2 N1 of the two-pass NTT worth timing for this ring (the default first).
int ntt_split_candidates(int logN, int* out, int cap);
void ntt_inverse(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off);
// The inverse NTT with row r's N^-1 replaced by scale[r] (a per-row constant times N^-1).
void ntt_inverse_scaled(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                        int mod_off, const ShoupPair* scale);

// Fast base conversion read by a forward NTT's first pass instead of its input: row r of item
// it (modulus m = mod_off + r) starts as sum_k y_k c_{k,m} mod m, with y_k the item's source
// limb k at src + it src_stride + k N (coefficient form, already multiplied by its inverse
// factor) and c_{k,m} = cst[k cst_s + m].  At most 8 source limbs.
struct BConvSrc {
    const uint64_t* src;
    size_t src_stride;
    const ShoupPair* cst;
    int cst_s;
    int ns;
};
void ntt_forward_bconv(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                       int mod_off, const BConvSrc& bc);

// The key switch's last step written by the row pass of that forward NTT instead of its
// output v: item z = 2 it + k, row m (modulus m): out = (u - v) P^-1 (+ c0[perm_g] for k = 0)
// (+ base), with u at u + z u_stride + m N and the per-it pointers outp / c0p / basep
// ([2][L][N] ciphertexts; c0p, basep may be null).  pinv[m] = P^-1 mod q_m.
struct CombineDst {
    const uint64_t* u;
    size_t u_stride;
    const uint64_t* const* c0p;
    const uint64_t* const* basep;
    uint64_t* const* outp;
    const ShoupPair* pinv;
    int L;
    uint32_t g;
};
void ntt_forward_bconv_combine(he_ctx* ctx, uint64_t* data, int items, size_t item_stride,
                               int rows, const BConvSrc& bc, const CombineDst& cd);
