// api.cu -- context, host-side tables and the C-ABI entry points (except the layer).
//
// Host arithmetic uses 128-bit integers.  Primes: deterministic Miller-Rabin.  Roots: the
// 2N-th root of a modulus m is x^((m-1)/2N) for the smallest quadratic non-residue x (for
// the plaintext modulus this root fixes the slot encoding).  Error sampler table: exact
// 128-bit fixed point (120 fractional bits).
#include <nvtx3/nvToolsExt.h>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "he_internal.cuh"
#include "eval.cuh"
#include "kernels.cuh"

// ------------------------------------------------------------------ host arithmetic

typedef unsigned __int128 u128;

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }

uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

uint64_t h_inv(uint64_t a, uint64_t q) { return h_powmod(a % q, q - 2, q); }

static bool h_is_prime(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : bases)
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : bases) {
        uint64_t x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

static bool gen_primes(int bits, int count, uint64_t two_n, const std::vector<uint64_t>& avoid,
                       std::vector<uint64_t>& out) {
    uint64_t top = (bits >= 64) ? ~0ull : ((1ull << bits) - 2);
    uint64_t p = (top / two_n) * two_n + 1;
    while ((int)out.size() < count) {
        if (p < two_n) return false;
        bool dup = false;
        for (uint64_t a : avoid) dup |= (a == p);
        if (!dup && h_is_prime(p)) out.push_back(p);
        p -= two_n;
    }
    return true;
}

static uint64_t root_2n(uint64_t q, uint64_t two_n) {
    uint64_t x = 2;
    while (h_powmod(x, (q - 1) / 2, q) != q - 1) ++x;
    return h_powmod(x, (q - 1) / two_n, q);
}

ShoupPair h_shoup(uint64_t w, uint64_t q) {
    return ShoupPair{w, (uint64_t)(((u128)w << 64) / q)};
}

uint64_t h_to_mont(uint64_t x, uint64_t q) { return (uint64_t)(((u128)(x % q) << 64) % q); }

static uint64_t mont_qinv_neg(uint64_t q) {
    uint64_t inv = q;  // q * q = 1 mod 8 for odd q
    for (int i = 0; i < 6; ++i) inv *= 2 - q * inv;
    return (uint64_t)0 - inv;
}

static uint32_t h_brv(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int b = 0; b < bits; ++b)
        if (x & (1u << b)) r |= 1u << (bits - 1 - b);
    return r;
}

// ---- multi-word unsigned integers (little-endian 64-bit words)

void mw_mul_small(std::vector<uint64_t>& a, uint64_t m) {
    uint64_t carry = 0;
    for (auto& w : a) {
        u128 p = (u128)w * m + carry;
        w = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
    if (carry) a.push_back(carry);
}

uint64_t mw_mod_small(const std::vector<uint64_t>& a, uint64_t m) {
    u128 r = 0;
    for (size_t i = a.size(); i-- > 0;) r = ((r << 64) | a[i]) % m;
    return (uint64_t)r;
}

std::vector<uint64_t> mw_div_small(const std::vector<uint64_t>& a, uint64_t m) {
    std::vector<uint64_t> q(a.size());
    u128 r = 0;
    for (size_t i = a.size(); i-- > 0;) {
        u128 cur = (r << 64) | a[i];
        q[i] = (uint64_t)(cur / m);
        r = cur % m;
    }
    while (q.size() > 1 && q.back() == 0) q.pop_back();
    return q;
}

// ---- error sampler table in 128-bit fixed point (F = 120 fractional bits)

namespace {
constexpr int FX = 120;

u128 fx_mul(u128 a, u128 b) {  // (a * b) >> FX, exact floor, a, b < 2^125
    uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    // 256-bit sum as four words
    uint64_t w[4] = {0, 0, 0, 0};
    auto add_at = [&](int pos, u128 v) {
        u128 s = (u128)w[pos] + (uint64_t)v;
        w[pos] = (uint64_t)s;
        u128 carry = (s >> 64) + (v >> 64);
        for (int k = pos + 1; k < 4 && carry; ++k) {
            u128 t = (u128)w[k] + (uint64_t)carry;
            w[k] = (uint64_t)t;
            carry = (t >> 64) + (carry >> 64);
        }
    };
    add_at(0, p00);
    add_at(1, p01);
    add_at(1, p10);
    add_at(2, p11);
    // shift right by 120 = 64 + 56
    u128 lo = ((u128)w[1] >> 56) | ((u128)w[2] << 8) | ((u128)w[3] << 72);
    return lo;
}

u128 fx_pow(u128 base, uint64_t e) {
    u128 r = (u128)1 << FX;
    while (e) {
        if (e & 1) r = fx_mul(r, base);
        base = fx_mul(base, base);
        e >>= 1;
    }
    return r;
}
}  // namespace

// T[m] = floor(2^63 Pr(|e| <= m)) for the discrete Gaussian rho(x) = exp(-x^2 / (2 sigma^2)),
// sigma = 3.2 (2 sigma^2 = 512/25), |e| <= 19.  exp(-25 m^2 / 512) = c^(25 m^2) with
// c = exp(-1/512) from its Taylor series.
void he_cdt_compute(uint64_t out[20]) {
    const u128 one = (u128)1 << FX;
    const u128 x = one >> 9;  // 1/512
    u128 pos = one, neg = 0, term = one;
    for (int k = 1; k < 40; ++k) {
        term = fx_mul(term, x) / (u128)k;
        if (k & 1) neg += term;
        else pos += term;
    }
    const u128 c = pos - neg;
    u128 rho[20];
    for (int m = 0; m < 20; ++m) rho[m] = fx_pow(c, 25ull * m * m);
    u128 z = rho[0];
    for (int m = 1; m < 20; ++m) z += 2 * rho[m];
    u128 acc = 0;
    for (int m = 0; m < 19; ++m) {
        acc += (m == 0) ? rho[0] : 2 * rho[m];
        u128 r = acc;
        uint64_t qv = 0;
        for (int b = 0; b < 63; ++b) {
            r <<= 1;
            qv <<= 1;
            if (r >= z) {
                r -= z;
                qv |= 1;
            }
        }
        out[m] = qv;
    }
    out[19] = 1ull << 63;
}

// ---- SplitMix64 stream start (same definition the kernels use for the draws)

static uint64_t h_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t he_stream_state(uint64_t seed, uint64_t stream) { return h_mix64(seed ^ h_mix64(stream)); }

// ------------------------------------------------------------------ context plumbing

int he_fail(he_ctx* ctx, int code, const std::string& msg) {
    if (ctx) {
        ctx->err = msg;
        // any failure while recording spoils the recording (a call may have recorded part of
        // its work before failing): he_graph_end then discards it
        if (ctx->rec && !ctx->rec->failed) ctx->rec->failed = code;
    }
    return code;
}

int check_device_error(he_ctx* ctx) {
    int word = 0;
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    HE_CHECK_CUDA(ctx, cudaMemcpy(&word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (word) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return he_fail(ctx, HE_ETIMEOUT, "a bounded device wait ran out: results since the last "
                                         "check are unusable");
    }
    return HE_OK;
}

extern "C" int he_check(he_ctx* ctx) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_check");
    HE_CHECK_CUDA(ctx, cudaGetLastError());
    return check_device_error(ctx);
}

int he_launch_check(he_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return he_fail(ctx, HE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return HE_OK;
}

static int refuse_growth(he_ctx* ctx) {
    return he_fail(ctx, HE_EINVAL, "a recorded call needs more scratch than the context holds: "
                                   "run the same calls once before he_graph_begin");
}

int arena_reserve(he_ctx* ctx, size_t n_u64) {
    size_t bytes = n_u64 * 8 + 4096;
    if (bytes <= ctx->arena.cap) return HE_OK;
    if (ctx->rec) return refuse_growth(ctx);
    if (ctx->arena.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->arena.base);
        ctx->arena.base = nullptr;
        ctx->arena.cap = 0;
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&ctx->arena.base, want) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "scratch allocation of " + std::to_string(want) + " bytes failed");
    }
    ctx->arena.cap = want;
    ++ctx->arena_epoch;
    return HE_OK;
}

int net_reserve(he_ctx* ctx, size_t n_u64) {
    const size_t bytes = n_u64 * 8 + 4096;
    if (bytes <= ctx->net.cap) return HE_OK;
    if (ctx->rec) return refuse_growth(ctx);
    if (ctx->net.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->net.base);
        ctx->net.base = nullptr;
        ctx->net.cap = 0;
    }
    if (cudaMalloc(&ctx->net.base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "network buffer allocation failed");
    }
    ctx->net.cap = bytes;
    ++ctx->net_epoch;
    return HE_OK;
}

int pk_reserve(he_ctx* ctx, size_t n_u64) {
    const size_t bytes = n_u64 * 8 + 4096;
    if (bytes <= ctx->pk.cap) return HE_OK;
    if (ctx->rec) return refuse_growth(ctx);
    if (ctx->pk.base) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->pk.base);
        ctx->pk.base = nullptr;
        ctx->pk.cap = 0;
    }
    if (cudaMalloc(&ctx->pk.base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "tap product buffer allocation failed");
    }
    ctx->pk.cap = bytes;
    ++ctx->pk_epoch;
    return HE_OK;
}

void arena_reset(he_ctx* ctx) { ctx->arena.used = 0; }

uint64_t* arena_take(he_ctx* ctx, size_t n_u64) {
    size_t bytes = (n_u64 * 8 + 255) & ~(size_t)255;
    if (ctx->arena.used + bytes > ctx->arena.cap) return nullptr;
    uint64_t* p = (uint64_t*)(ctx->arena.base + ctx->arena.used);
    ctx->arena.used += bytes;
    return p;
}

// Small host->device uploads go through a ring of pinned staging slots so that they stay
// asynchronous; a slot is reused only after the copy that last read it has executed.
const void* upload_small(he_ctx* ctx, const void* src, size_t bytes) {
    if (ctx->rec) {                              // recording a graph: a buffer the graph owns
        void* d = nullptr;
        if (cudaMalloc(&d, bytes ? bytes : 8) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->rec->g.allocs.push_back(d);
        if (bytes && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return d;
    }
    Staging& st = ctx->staging;
    if (bytes > st.slot_bytes) return nullptr;
    int slot = st.next;
    st.next = (st.next + 1) % st.n_slots;
    cudaEventSynchronize(st.ev[slot]);
    char* h = st.host + (size_t)slot * st.slot_bytes;
    char* d = st.dev + (size_t)slot * st.slot_bytes;
    memcpy(h, src, bytes);
    if (cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return nullptr;
    cudaEventRecord(st.ev[slot], ctx->stream);
    return d;
}

// Host -> device copy of call arguments into device memory the call owns (scratch): an
// ordinary asynchronous copy, or, while a graph is recorded, a copy into a device buffer the
// graph owns plus a recorded device-to-device copy (a replay must not read host memory that
// belonged to the recorded call).
int upload_host(he_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (!bytes) return HE_OK;
    if (ctx->rec) {
        void* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
            cudaGetLastError();
            return he_fail(ctx, HE_ENOMEM, "table allocation while recording failed");
        }
        ctx->rec->g.allocs.push_back(d);
        HE_CHECK_CUDA(ctx, cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return HE_OK;
    }
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return HE_OK;
}

// Call arguments to the device: through a pinned staging slot when they fit (asynchronous),
// else into `scratch` (device memory of the caller's) with upload_host, whose copy from
// pageable memory waits for the stream first.  Returns the device copy or NULL.
const void* upload_args(he_ctx* ctx, const void* src, size_t bytes, void* scratch) {
    if (bytes <= ctx->staging.slot_bytes) return upload_small(ctx, src, bytes);
    if (!scratch || upload_host(ctx, scratch, src, bytes)) return nullptr;
    return scratch;
}

uint32_t galois_elt(const he_ctx* ctx, int32_t step) {
    const uint64_t two_n = 2ull * ctx->N;
    if (step == HE_ROW_SWAP) return (uint32_t)(two_n - 1);
    if (step == HE_RELIN_KEY) return 0u;          // the s^2 -> s key lives in slot 0
    int64_t half = ctx->N / 2;
    int64_t k = ((int64_t)step % half + half) % half;
    return (uint32_t)h_powmod(5, (uint64_t)k, two_n);
}

template <typename T>
static int upload_vec(he_ctx* ctx, T** dptr, const std::vector<T>& v) {
    if (v.empty()) {
        *dptr = nullptr;
        return HE_OK;
    }
    if (cudaMalloc((void**)dptr, v.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "table allocation failed");
    }
    if (cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return he_fail(ctx, HE_ECUDA, "table upload failed");
    return HE_OK;
}

static void free_ctx(he_ctx* c) {
    if (!c) return;
    recording_abort(c);
    if (c->stream || true) cudaStreamSynchronize(c->stream);
    void* ptrs[] = {c->d_mod, c->d_tw_fwd, c->d_tw_inv, c->d_tw_fwd_rows, c->d_slot_pos, c->d_cdt,
                    c->d_modup_inv, c->d_modup_c, c->d_md_inv, c->d_md_c, c->d_md_pinv,
                    c->d_modup_ninv, c->d_md_ninv,
                    c->d_rs_inv, c->d_pmodq, c->arena.base, c->staging.dev, c->d_err,
                    c->d_mult_tab, c->net.base, c->pk.base};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& kv : c->keys)
        if (kv.second.dev) cudaFree(kv.second.dev);
    for (auto& kv : c->plans)
        if (kv.second.pts) cudaFree(kv.second.pts);
    for (auto& kv : c->graphs) graph_release(kv.second);
    if (c->staging.host) cudaFreeHost(c->staging.host);
    for (auto e : c->staging.ev)
        if (e) cudaEventDestroy(e);
    for (auto& sp : c->spans) {
        cudaEventDestroy(sp.a);
        cudaEventDestroy(sp.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
}

// ------------------------------------------------------------------ context creation

extern "C" int he_ctx_create(const he_params* p, void* stream, he_ctx** out) {
    if (!out) return HE_EINVAL;
    *out = nullptr;
    if (!p) return HE_EINVAL;
    if (p->log_n < 6 || p->log_n > 16 || p->n_q < 1 || p->n_q > 32 || p->n_p < 1 || p->n_p > 8 ||
        p->q_bits < 20 || p->q_bits > 60 || p->p_bits < 20 || p->p_bits > 60 || p->alpha < 1 ||
        p->alpha > p->n_q || p->alpha > 8 || p->t < 3 || p->t >= (1ull << 62) || !(p->t & 1) ||
        !h_is_prime(p->t))
        return HE_EINVAL;
    he_ctx* c = new he_ctx();
    c->prm = *p;
    c->stream = (cudaStream_t)stream;
    c->logN = p->log_n;
    c->N = 1 << p->log_n;
    c->L = p->n_q;
    c->K = p->n_p;
    c->alpha = p->alpha;
    c->dnum = (c->L + c->alpha - 1) / c->alpha;
    // auxiliary basis for ciphertext products: prod B > N Q (60-bit primes, ~59.9 bits each)
    c->n_b = (int)((c->L * p->q_bits + p->log_n + 4 + 58) / 59);
    c->n_mod = c->L + c->K + 1 + c->n_b;
    const uint64_t two_n = 2ull * c->N;
    std::vector<uint64_t> qs, ps, bs;
    if (!gen_primes(p->q_bits, c->L, two_n, {}, qs) || !gen_primes(p->p_bits, c->K, two_n, qs, ps)) {
        delete c;
        return HE_EINVAL;
    }
    {
        std::vector<uint64_t> avoid = qs;
        avoid.insert(avoid.end(), ps.begin(), ps.end());
        avoid.push_back(p->t);
        if (!gen_primes(60, c->n_b, two_n, avoid, bs)) {
            delete c;
            return HE_EINVAL;
        }
    }
    c->mods = qs;
    c->mods.insert(c->mods.end(), ps.begin(), ps.end());
    c->mods.push_back(p->t);
    c->mods.insert(c->mods.end(), bs.begin(), bs.end());
    c->batching = ((p->t - 1) % two_n) == 0;
    const int N = c->N, L = c->L, K = c->K, LK = L + K;

    // per-modulus constants and twiddles (the plaintext modulus only when it has a 2N-th root)
    std::vector<ModConst> mc(c->n_mod);
    std::vector<ShoupPair> twf((size_t)c->n_mod * N), twi((size_t)c->n_mod * N);
    for (int m = 0; m < c->n_mod; ++m) {
        uint64_t q = c->mods[m];
        ModConst& M = mc[m];
        M.q = q;
        M.qinv_neg = mont_qinv_neg(q);
        uint64_t r1 = (uint64_t)(((u128)1 << 64) % q);
        M.r2 = h_mulmod(r1, r1, q);
        M.n_inv = h_inv((uint64_t)N % q, q);
        M.n_inv_sh = h_shoup(M.n_inv, q).ws;
        M.one_sh = h_shoup(1, q).ws;
        if ((q >> 57) == 0) {
            const int b = 64 - __builtin_clzll(q);
            M.red_sh = (uint16_t)std::max(b - 25, 0);
            M.red_t = (uint16_t)(31 + b - M.red_sh);
            M.red_r = (uint32_t)(((u128)1 << (31 + b)) / q);
        }
        if (m == c->L + c->K && !c->batching) continue;   // t without a 2N-th root
        uint64_t psi = root_2n(q, two_n), psi_inv = h_inv(psi, q);
        for (int k = 0; k < N; ++k) {
            uint32_t e = h_brv((uint32_t)k, c->logN);
            twf[(size_t)m * N + k] = h_shoup(h_powmod(psi, e, q), q);
            twi[(size_t)m * N + k] = h_shoup(h_powmod(psi_inv, e, q), q);
        }
    }
    // slot -> NTT position (slot j of row 0 evaluates at zeta^(5^j), row 1 at zeta^(-5^j))
    std::vector<int32_t> pos(N, 0);
    {
        uint64_t x = 1;
        for (int j = 0; j < N / 2; ++j) {
            uint64_t e0 = x, e1 = (two_n - x) % two_n;
            pos[j] = (int32_t)h_brv((uint32_t)((e0 - 1) / 2), c->logN);
            pos[N / 2 + j] = (int32_t)h_brv((uint32_t)((e1 - 1) / 2), c->logN);
            x = x * 5 % two_n;
        }
    }
    uint64_t cdt[20];
    he_cdt_compute(cdt);
    std::vector<uint64_t> cdtv(cdt, cdt + 20);

    // ModUp constants
    std::vector<ShoupPair> mu_inv(L), mu_c((size_t)c->dnum * c->alpha * LK, ShoupPair{0, 0});
    for (int j = 0; j < c->dnum; ++j) {
        int i0 = j * c->alpha, i1 = std::min(i0 + c->alpha, L);
        for (int i = i0; i < i1; ++i) {
            uint64_t qi = qs[i];
            uint64_t prod_qi = 1;
            for (int k = i0; k < i1; ++k)
                if (k != i) prod_qi = h_mulmod(prod_qi, qs[k] % qi, qi);
            mu_inv[i] = h_shoup(h_inv(prod_qi, qi), qi);
            for (int l = 0; l < LK; ++l) {
                uint64_t ml = c->mods[l], v = 1;
                for (int k = i0; k < i1; ++k)
                    if (k != i) v = h_mulmod(v, qs[k] % ml, ml);
                mu_c[((size_t)j * c->alpha + (i - i0)) * LK + l] = h_shoup(v, ml);
            }
        }
    }
    // ModDown constants
    std::vector<ShoupPair> md_inv(K), md_c((size_t)K * L), md_pinv(L);
    std::vector<uint64_t> pmodq(L);
    for (int k = 0; k < K; ++k) {
        uint64_t pk = ps[k], v = 1;
        for (int kk = 0; kk < K; ++kk)
            if (kk != k) v = h_mulmod(v, ps[kk] % pk, pk);
        md_inv[k] = h_shoup(h_inv(v, pk), pk);
        for (int i = 0; i < L; ++i) {
            uint64_t qi = qs[i], w = 1;
            for (int kk = 0; kk < K; ++kk)
                if (kk != k) w = h_mulmod(w, ps[kk] % qi, qi);
            md_c[(size_t)k * L + i] = h_shoup(w, qi);
        }
    }
    for (int i = 0; i < L; ++i) {
        uint64_t qi = qs[i], P = 1;
        for (int k = 0; k < K; ++k) P = h_mulmod(P, ps[k] % qi, qi);
        md_pinv[i] = h_shoup(h_inv(P, qi), qi);
        pmodq[i] = h_to_mont(P, qi);
    }
    std::vector<ShoupPair> mu_ninv(L), md_ninv(K);
    for (int i = 0; i < L; ++i) mu_ninv[i] = h_shoup(h_mulmod(mc[i].n_inv, mu_inv[i].w, qs[i]), qs[i]);
    for (int k = 0; k < K; ++k) md_ninv[k] = h_shoup(h_mulmod(mc[L + k].n_inv, md_inv[k].w, ps[k]), ps[k]);
    std::vector<ShoupPair> rs((size_t)L * L, ShoupPair{0, 0});
    for (int lv = 1; lv < L; ++lv)
        for (int i = 0; i < lv; ++i) rs[(size_t)lv * L + i] = h_shoup(h_inv(qs[lv] % qs[i], qs[i]), qs[i]);

    int rc = HE_OK;
    if ((rc = upload_vec(c, &c->d_mod, mc)) || (rc = upload_vec(c, &c->d_tw_fwd, twf)) ||
        (rc = upload_vec(c, &c->d_tw_inv, twi)) || (rc = upload_vec(c, &c->d_tw_fwd_rows, twf)) ||
        (rc = upload_vec(c, &c->d_slot_pos, pos)) ||
        (rc = upload_vec(c, &c->d_cdt, cdtv)) || (rc = upload_vec(c, &c->d_modup_inv, mu_inv)) ||
        (rc = upload_vec(c, &c->d_modup_c, mu_c)) || (rc = upload_vec(c, &c->d_md_inv, md_inv)) ||
        (rc = upload_vec(c, &c->d_md_c, md_c)) || (rc = upload_vec(c, &c->d_md_pinv, md_pinv)) ||
        (rc = upload_vec(c, &c->d_modup_ninv, mu_ninv)) || (rc = upload_vec(c, &c->d_md_ninv, md_ninv)) ||
        (rc = upload_vec(c, &c->d_rs_inv, rs)) || (rc = upload_vec(c, &c->d_pmodq, pmodq))) {
        free_ctx(c);
        return rc;
    }
    if (cudaMalloc((void**)&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return HE_ENOMEM;
    }
    Staging& st = c->staging;
    if (cudaMallocHost((void**)&st.host, st.slot_bytes * st.n_slots) != cudaSuccess ||
        cudaMalloc((void**)&st.dev, st.slot_bytes * st.n_slots) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return HE_ENOMEM;
    }
    for (int i = 0; i < st.n_slots; ++i) cudaEventCreateWithFlags(&st.ev[i], cudaEventDisableTiming);
    ntt_prepare(c);                             // row-pass twiddle order of the default split
    *out = c;
    return HE_OK;
}

extern "C" void he_ctx_destroy(he_ctx* ctx) { free_ctx(ctx); }

extern "C" const char* he_last_error(const he_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int he_set_stream(he_ctx* ctx, void* stream) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_set_stream");
    ctx->stream = (cudaStream_t)stream;
    return HE_OK;
}

extern "C" int he_get_moduli(const he_ctx* ctx, uint64_t* out, int cap) {
    const int n = ctx ? ctx->L + ctx->K + 1 : 0;
    if (!ctx || !out || cap < n) return HE_EINVAL;
    for (int i = 0; i < n; ++i) out[i] = ctx->mods[i];
    return n;
}

extern "C" void he_op_counts(const he_ctx* ctx, uint64_t out[4]) {
    for (int i = 0; i < 4; ++i) out[i] = ctx ? ctx->ops[i] : 0;
}

extern "C" void he_reset_op_counts(he_ctx* ctx) {
    if (ctx)
        for (int i = 0; i < 4; ++i) ctx->ops[i] = 0;
}

extern "C" void he_gaussian_table(uint64_t out[20]) { he_cdt_compute(out); }

extern "C" uint64_t he_launch_count(const he_ctx* ctx) { return ctx ? ctx->launches : 0; }

static const char* const kPhaseNames[HE_N_PHASES] = {"encode", "modup", "taps", "moddown",
                                                     "rotate", "restore", "multiply", "phase7"};

void phase_begin(he_ctx* ctx, int phase) {
    if (ctx->nvtx_open) nvtxRangeEnd(ctx->nvtx_id);       // a phase left by an error return
    ctx->nvtx_id = nvtxRangeStartA(phase >= 0 && phase < HE_N_PHASES ? kPhaseNames[phase] : "phase");
    ctx->nvtx_open = true;
    if (!ctx->timing) return;
    he_ctx::PhaseSpan sp{phase, nullptr, nullptr};
    for (cudaEvent_t* e : {&sp.a, &sp.b}) {
        if (!ctx->event_pool.empty()) {
            *e = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    cudaEventRecord(sp.a, ctx->stream);
    ctx->spans.push_back(sp);
}

void phase_end(he_ctx* ctx) {
    if (ctx->nvtx_open) {
        nvtxRangeEnd(ctx->nvtx_id);
        ctx->nvtx_open = false;
    }
    if (!ctx->timing || ctx->spans.empty()) return;
    cudaEventRecord(ctx->spans.back().b, ctx->stream);
}

extern "C" int he_set_phase_timing(he_ctx* ctx, int enable) {
    if (!ctx) return HE_EINVAL;
    ctx->timing = enable != 0;
    return HE_OK;
}

extern "C" int he_phase_times(he_ctx* ctx, double* ms_out, uint64_t* calls_out) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_phase_times");
    int rc = check_device_error(ctx);
    if (rc) return rc;
    for (auto& sp : ctx->spans) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess && sp.phase >= 0 &&
            sp.phase < HE_N_PHASES) {
            ctx->phase_ms[sp.phase] += ms;
            ctx->phase_calls[sp.phase] += 1;
        }
        cudaGetLastError();
        ctx->event_pool.push_back(sp.a);
        ctx->event_pool.push_back(sp.b);
    }
    ctx->spans.clear();
    for (int i = 0; i < HE_N_PHASES; ++i) {
        if (ms_out) ms_out[i] = ctx->phase_ms[i];
        if (calls_out) calls_out[i] = ctx->phase_calls[i];
        ctx->phase_ms[i] = 0;
        ctx->phase_calls[i] = 0;
    }
    return HE_OK;
}

// ------------------------------------------------------------------ validation helpers

int check_ct(he_ctx* ctx, const he_ct* ct, int need_limbs, int need_domain, const char* what) {
    if (!ct || !ct->data) return he_fail(ctx, HE_EINVAL, std::string(what) + ": null ciphertext");
    if (ct->n_polys != 2) return he_fail(ctx, HE_EINVAL, std::string(what) + ": n_polys must be 2");
    if (ct->n_limbs < 1 || (int)ct->n_limbs > ctx->L)
        return he_fail(ctx, HE_EINVAL, std::string(what) + ": bad n_limbs");
    if (need_limbs > 0 && (int)ct->n_limbs != need_limbs)
        return he_fail(ctx, HE_EINVAL, std::string(what) + ": wrong level");
    if (need_domain >= 0 && ct->domain != need_domain)
        return he_fail(ctx, HE_EINVAL, std::string(what) + ": wrong domain");
    return HE_OK;
}

// ------------------------------------------------------------------ representation

extern "C" int he_to_ntt(he_ctx* ctx, he_ct* ct) {
    if (!ctx) return HE_EINVAL;
    int rc = check_ct(ctx, ct, 0, HE_COEFF, "he_to_ntt");
    if (rc) return rc;
    ntt_forward(ctx, ct->data, 2, (size_t)ct->n_limbs * ctx->N, ct->n_limbs, 0);
    ct->domain = HE_NTT;
    return he_launch_check(ctx, "he_to_ntt");
}

extern "C" int he_to_coeff(he_ctx* ctx, he_ct* ct) {
    if (!ctx) return HE_EINVAL;
    int rc = check_ct(ctx, ct, 0, HE_NTT, "he_to_coeff");
    if (rc) return rc;
    ntt_inverse(ctx, ct->data, 2, (size_t)ct->n_limbs * ctx->N, ct->n_limbs, 0);
    ct->domain = HE_COEFF;
    return he_launch_check(ctx, "he_to_coeff");
}

extern "C" int he_ntt(he_ctx* ctx, uint64_t* data, int n_items, int n_limbs, int inverse) {
    if (!ctx || !data || n_items < 1 || n_limbs < 1 || n_limbs > ctx->L + ctx->K)
        return ctx ? he_fail(ctx, HE_EINVAL, "he_ntt: bad arguments") : HE_EINVAL;
    if (inverse) ntt_inverse(ctx, data, n_items, (size_t)n_limbs * ctx->N, n_limbs, 0);
    else ntt_forward(ctx, data, n_items, (size_t)n_limbs * ctx->N, n_limbs, 0);
    return he_launch_check(ctx, "he_ntt");
}

// Encode slot values already on the device (items x N int64) into plaintexts [items][L][N]
// (centred lift, NTT domain; Montgomery form when mont != 0).  `tmp` holds items x N u64.
void encode_device(he_ctx* ctx, const int64_t* d_slots, int items, uint64_t* tmp, uint64_t* out,
                   int mont, int rows) {
    launch_slots_to_ntt(ctx, d_slots, tmp, items);
    ntt_inverse(ctx, tmp, items, (size_t)ctx->N, 1, ctx->L + ctx->K);
    launch_lift(ctx, tmp, out, items, rows, mont);
    ntt_forward(ctx, out, items, (size_t)rows * ctx->N, rows, 0);
}

extern "C" int he_encode(he_ctx* ctx, const int64_t* slots, uint64_t* pt_out) {
    if (!ctx || !slots || !pt_out) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_encode");
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_encode: t is not 1 mod 2N");
    const size_t N = ctx->N;
    int rc = arena_reserve(ctx, 2 * N);
    if (rc) return rc;
    arena_reset(ctx);
    int64_t* ds = (int64_t*)arena_take(ctx, N);
    uint64_t* tmp = arena_take(ctx, N);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(ds, slots, N * 8, cudaMemcpyHostToDevice, ctx->stream));
    encode_device(ctx, ds, 1, tmp, pt_out, 0, ctx->L);
    rc = he_launch_check(ctx, "he_encode");
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return rc;
}

// ------------------------------------------------------------------ client side

// s (host int64[N]) -> residues over `rows` moduli from index 0, NTT domain; Montgomery copy
// in s_m when non-null.
static void secret_to_device(he_ctx* ctx, const int64_t* d_sk, int rows, uint64_t* s_ntt,
                             uint64_t* s_m) {
    launch_from_signed(ctx, d_sk, s_ntt, rows, 0);
    ntt_forward(ctx, s_ntt, 1, 0, rows, 0);
    if (s_m) {
        cudaMemcpyAsync(s_m, s_ntt, (size_t)rows * ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->stream);
        launch_to_mont(ctx, s_m, 1, rows, rows + ctx->K + 1, 0);
    }
}

extern "C" int he_keygen_secret(he_ctx* ctx, uint64_t seed, int64_t* sk_out) {
    if (!ctx || !sk_out) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_keygen_secret");
    int rc = arena_reserve(ctx, ctx->N);
    if (rc) return rc;
    arena_reset(ctx);
    int64_t* d = (int64_t*)arena_take(ctx, ctx->N);
    launch_ternary(ctx, he_stream_state(seed, 1), d);
    if ((rc = he_launch_check(ctx, "he_keygen_secret"))) return rc;
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(sk_out, d, (size_t)ctx->N * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HE_OK;
}

extern "C" int he_encrypt(he_ctx* ctx, const int64_t* sk, const int64_t* slots, uint64_t seed,
                          he_ct* out) {
    if (!ctx || !sk || !slots) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_encrypt");
    int rc = check_ct(ctx, out, ctx->L, -1, "he_encrypt");
    if (rc) return rc;
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_encrypt: t is not 1 mod 2N");
    if (out->domain != HE_COEFF && out->domain != HE_NTT) return he_fail(ctx, HE_EINVAL, "he_encrypt: domain");
    const size_t N = ctx->N, L = ctx->L;
    if ((rc = arena_reserve(ctx, 5 * N + 3 * L * N))) return rc;
    arena_reset(ctx);
    int64_t* d_sk = (int64_t*)arena_take(ctx, N);
    int64_t* d_sl = (int64_t*)arena_take(ctx, N);
    int64_t* d_e = (int64_t*)arena_take(ctx, N);
    uint64_t* m = arena_take(ctx, N);
    uint64_t* tmp = arena_take(ctx, N);
    uint64_t* s_ntt = arena_take(ctx, L * N);
    uint64_t* s_m = arena_take(ctx, L * N);
    uint64_t* as = arena_take(ctx, L * N);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(d_sk, sk, N * 8, cudaMemcpyHostToDevice, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(d_sl, slots, N * 8, cudaMemcpyHostToDevice, ctx->stream));
    // m = encoding of the slots, coefficients in [0, t)
    launch_slots_to_ntt(ctx, d_sl, m, 1);
    ntt_inverse(ctx, m, 1, N, 1, ctx->L + ctx->K);
    secret_to_device(ctx, d_sk, (int)L, s_ntt, s_m);
    uint64_t* c0 = out->data;
    uint64_t* c1 = out->data + L * N;
    launch_uniform(ctx, he_stream_state(seed, 2), c1, (int)L, 0, 0);   // a, coefficient form
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(as, c1, L * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    ntt_forward(ctx, as, 1, 0, (int)L, 0);
    launch_dec_phase_mul(ctx, as, s_m, (int)L);                            // as <- a * s
    ntt_inverse(ctx, as, 1, 0, (int)L, 0);
    launch_gaussian(ctx, he_stream_state(seed, 3), d_e);
    // Delta_i = floor(Q / t) mod q_i
    std::vector<uint64_t> Q{1};
    for (size_t i = 0; i < L; ++i) mw_mul_small(Q, ctx->mods[i]);
    std::vector<uint64_t> D = mw_div_small(Q, ctx->prm.t);
    std::vector<ShoupPair> dl(L);
    for (size_t i = 0; i < L; ++i) dl[i] = h_shoup(mw_mod_small(D, ctx->mods[i]), ctx->mods[i]);
    const ShoupPair* d_dl = (const ShoupPair*)upload_small(ctx, dl.data(), L * sizeof(ShoupPair));
    if (!d_dl) return he_fail(ctx, HE_ECUDA, "he_encrypt: upload failed");
    launch_enc_c0(ctx, d_e, m, as, d_dl, c0);
    if (out->domain == HE_NTT) ntt_forward(ctx, out->data, 2, L * N, (int)L, 0);
    (void)tmp;
    rc = he_launch_check(ctx, "he_encrypt");
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return rc;
}

extern "C" int he_decrypt(he_ctx* ctx, const int64_t* sk, const he_ct* ct, int64_t* slots_out) {
    if (!ctx || !sk || !slots_out) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_decrypt");
    int rc = check_ct(ctx, ct, 0, -1, "he_decrypt");
    if (rc) return rc;
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_decrypt: t is not 1 mod 2N");
    const size_t N = ctx->N, Lv = ct->n_limbs;
    // constants of level Lv: [(Q/q_i)^-1]_{q_i} (Shoup), Q/q_i and Q as W-word integers
    std::vector<uint64_t> Q{1};
    for (size_t i = 0; i < Lv; ++i) mw_mul_small(Q, ctx->mods[i]);
    const int W = (int)Q.size();
    if (W > HE_DEC_MAX_WORDS) return he_fail(ctx, HE_EINVAL, "he_decrypt: modulus too large");
    std::vector<uint64_t> cst(2 * Lv + Lv * W + W, 0);
    for (size_t i = 0; i < Lv; ++i) {
        uint64_t qi = ctx->mods[i], v = 1;
        std::vector<uint64_t> qh{1};
        for (size_t k = 0; k < Lv; ++k)
            if (k != i) {
                v = h_mulmod(v, ctx->mods[k] % qi, qi);
                mw_mul_small(qh, ctx->mods[k]);
            }
        ShoupPair sp = h_shoup(h_inv(v, qi), qi);
        cst[2 * i] = sp.w;
        cst[2 * i + 1] = sp.ws;
        for (int w = 0; w < W && w < (int)qh.size(); ++w) cst[2 * Lv + i * W + w] = qh[w];
    }
    for (int w = 0; w < W; ++w) cst[2 * Lv + Lv * W + w] = Q[w];
    if ((rc = arena_reserve(ctx, 6 * N + 4 * Lv * N + cst.size()))) return rc;
    arena_reset(ctx);
    int64_t* d_sk = (int64_t*)arena_take(ctx, N);
    uint64_t* X = arena_take(ctx, 2 * Lv * N);
    uint64_t* s_ntt = arena_take(ctx, Lv * N);
    uint64_t* s_m = arena_take(ctx, Lv * N);
    uint64_t* m = arena_take(ctx, N);
    int64_t* d_out = (int64_t*)arena_take(ctx, N);
    uint64_t* d_cst = arena_take(ctx, cst.size());
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(d_sk, sk, N * 8, cudaMemcpyHostToDevice, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(d_cst, cst.data(), cst.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X, ct->data, 2 * Lv * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ct->domain == HE_COEFF) ntt_forward(ctx, X, 2, Lv * N, (int)Lv, 0);
    secret_to_device(ctx, d_sk, (int)Lv, s_ntt, s_m);
    launch_dec_phase(ctx, X, s_m, X, (int)Lv);   // X[0] <- c0 + c1 s
    ntt_inverse(ctx, X, 1, 0, (int)Lv, 0);
    launch_dec_round(ctx, X, m, (int)Lv, W, d_cst);
    ntt_forward(ctx, m, 1, 0, 1, ctx->L + ctx->K);
    launch_ntt_to_slots(ctx, m, d_out, 1);
    if ((rc = he_launch_check(ctx, "he_decrypt"))) return rc;
    if ((rc = check_device_error(ctx))) return rc;
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(slots_out, d_out, N * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HE_OK;
}

// ------------------------------------------------------------------ Galois keys

extern "C" int he_keygen_galois(he_ctx* ctx, const int64_t* sk, uint64_t seed,
                                const int32_t* steps, int n_steps) {
    if (!ctx || !sk || (n_steps > 0 && !steps) || n_steps < 0) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_keygen_galois");
    const size_t N = ctx->N, LK = ctx->L + ctx->K;
    int rc = arena_reserve(ctx, 2 * N + 4 * LK * N);
    if (rc) return rc;
    arena_reset(ctx);
    int64_t* d_sk = (int64_t*)arena_take(ctx, N);
    int64_t* d_e = (int64_t*)arena_take(ctx, N);
    uint64_t* s_ntt = arena_take(ctx, LK * N);
    uint64_t* s_m = arena_take(ctx, LK * N);
    uint64_t* sg = arena_take(ctx, LK * N);
    uint64_t* E = arena_take(ctx, LK * N);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(d_sk, sk, N * 8, cudaMemcpyHostToDevice, ctx->stream));
    launch_from_signed(ctx, d_sk, s_ntt, (int)LK, 0);
    ntt_forward(ctx, s_ntt, 1, 0, (int)LK, 0);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(s_m, s_ntt, LK * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    launch_to_mont(ctx, s_m, 1, (int)LK, (int)LK + 1, 0);
    for (int si = 0; si < n_steps; ++si) {
        uint32_t g = galois_elt(ctx, steps[si]);
        uint64_t* key = nullptr;
        if ((rc = he_key_for_generation(ctx, g, &key))) return rc;
        const bool relin = g == 0u;
        if (relin) {   // target s^2 (NTT domain: s_ntt * s_ntt)
            HE_CHECK_CUDA(ctx, cudaMemcpyAsync(sg, s_ntt, LK * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            launch_dec_phase_mul(ctx, sg, s_m, (int)LK);
        } else {
            launch_automorph(ctx, s_ntt, 0, sg, 0, 1, (int)LK, g);   // s(X^g), NTT domain
        }
        for (int j = 0; j < ctx->dnum; ++j) {
            uint64_t* b = key + (size_t)(2 * j) * LK * N;
            uint64_t* a = key + (size_t)(2 * j + 1) * LK * N;
            const uint64_t sa = relin ? (6ull << 48) | (uint64_t)j
                                      : (4ull << 48) | ((uint64_t)g << 8) | (uint64_t)j;
            const uint64_t se = relin ? (7ull << 48) | (uint64_t)j
                                      : (5ull << 48) | ((uint64_t)g << 8) | (uint64_t)j;
            launch_uniform(ctx, he_stream_state(seed, sa), a, (int)LK, 0, 0);
            ntt_forward(ctx, a, 1, 0, (int)LK, 0);
            launch_gaussian(ctx, he_stream_state(seed, se), d_e);
            launch_from_signed(ctx, d_e, E, (int)LK, 0);
            ntt_forward(ctx, E, 1, 0, (int)LK, 0);
            int i0 = j * ctx->alpha, i1 = std::min(i0 + ctx->alpha, ctx->L);
            launch_keygen_b(ctx, a, s_m, E, sg, b, i0, i1);
            launch_to_mont(ctx, b, 1, (int)(2 * LK), (int)LK, 0);    // b and a are adjacent
        }
    }
    rc = he_launch_check(ctx, "he_keygen_galois");
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return rc;
}
