// mult.cu -- BFV ciphertext multiplication with relinearisation (the x^2 activation's core).
//
// out = Relin(round(t/Q (a0 + a1 s)(b0 + b1 s))): with a_k, b_k lifted to centred integers,
//   d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1   over Z[X]/(X^N+1),
//   d_k' = round(t d_k / Q) mod Q,  out = (d0' + u0, d1' + u1),  (u0, u1) = KeySwitch_{s^2 -> s}(d2').
// Exact throughout:
//   1. the centred lift of a_k to an auxiliary basis B (prod B > 16 N Q) is computed exactly
//      per coefficient (k_extend_exact): the CRT overflow count v = round(sum_i y_i / q_i)
//      comes from 128-bit fractions, or from the multi-word CRT value when those cannot
//      decide it;
//   2. the products are formed limb-wise over Q u B in the NTT domain (k_tensor), so d_k is
//      known modulo Q B > 32 |d_k|;
//   3. k_scale_round splits t d_k / Q into an integer known modulo each q_i and a small
//      fraction whose rounding the 128-bit fractions decide (multi-word long division when
//      they cannot).
// The relinearisation key is the switching key for s^2 (Galois element slot 0).
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

#define HE_MW_MAX 40   // 64-bit words of the largest multi-word value (Q B and its products)

namespace {

__device__ __forceinline__ int mw_cmp(const uint64_t* a, const uint64_t* b, int W) {
    for (int w = W - 1; w >= 0; --w)
        if (a[w] != b[w]) return a[w] > b[w] ? 1 : -1;
    return 0;
}

__device__ __forceinline__ void mw_sub(uint64_t* a, const uint64_t* b, int W) {   // a -= b
    uint64_t borrow = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t x = a[w], y = b[w];
        const uint64_t d = x - y - borrow;
        borrow = (x < y || (x == y && borrow)) ? 1u : 0u;
        a[w] = d;
    }
}

__device__ __forceinline__ void mw_mac(uint64_t* X, const uint64_t* A, int W, uint64_t s) {
    uint64_t carry = 0;                                   // X (W + 1 words) += A (W words) * s
    for (int w = 0; w < W; ++w) {
        unsigned __int128 p = (unsigned __int128)A[w] * s + X[w] + carry;
        X[w] = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
    }
    X[W] += carry;
}

__device__ __forceinline__ uint64_t mw_mod(const uint64_t* A, int W, uint64_t q) {
    unsigned __int128 r = 0;
    for (int w = W - 1; w >= 0; --w) r = ((r << 64) | A[w]) % q;
    return (uint64_t)r;
}

// 192-bit accumulator (w0 + w1 2^64 + w2 2^128 + w3 2^192) += y (fhi 2^64 + flo).
__device__ __forceinline__ void acc_mac192(uint64_t& w0, uint64_t& w1, uint64_t& w2, uint64_t& w3,
                                           uint64_t y, uint64_t fhi, uint64_t flo) {
    const uint64_t lo0 = y * flo, hi0 = mulhi64(y, flo);
    const uint64_t lo1 = y * fhi, hi1 = mulhi64(y, fhi);
    unsigned __int128 s = (unsigned __int128)w0 + lo0;
    w0 = (uint64_t)s;
    s >>= 64;
    s += (unsigned __int128)w1 + hi0 + lo1;
    w1 = (uint64_t)s;
    s >>= 64;
    s += (unsigned __int128)w2 + hi1;
    w2 = (uint64_t)s;
    s >>= 64;
    w3 += (uint64_t)s;
}

// The rounding of a sum of fractions decided from its fixed-point value: with S the exact sum
// and (w3, w2, w1, w0) a lower bound of it within 2^-64 (fraction words w1, w0), round(S) is
// w3 w2 + [w1 >= 2^63] unless w1 = 2^63 - 1, where the bound cannot separate S from 1/2.
constexpr uint64_t kNearHalf = 0x7fffffffffffffffull;

// Centred lift of a_k (coefficient form over Q, rows 0..L-1 of each item) to B (rows L..):
// x = sum_i y_i Qhat_i - v Q with y_i = [x_i Qhat_i^-1]_{q_i} and v = round(sum_i y_i / q_i),
// which puts x in (-Q/2, Q/2] (Q is odd, so the sum is never a half-integer); then
// x mod b_j = sum_i y_i [Qhat_i]_{b_j} - v [Q]_{b_j}.  v comes from the 128-bit fractions
// psi_i = floor(2^128 / q_i); when that bound is inconclusive (or force_exact is set) v is
// taken from the multi-word value of sum_i y_i Qhat_i instead.
// Tables (u64 words): exact: qhinv[L] pairs | Qhat[L][Wq] | Q[Wq+1] | qhat_b[L][nb] pairs |
// Q_b[nb] pairs; fast: psi[L] (hi, lo).
__global__ void k_extend_exact(uint64_t* __restrict__ data, size_t item_stride, int L, int nb,
                               int Wq, int b_off, int logN, const ModConst* __restrict__ mods,
                               const uint64_t* __restrict__ tab, const uint64_t* __restrict__ fast,
                               int force_exact) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    uint64_t* x = data + blockIdx.y * item_stride;
    const uint64_t* qhinv = tab;
    const uint64_t* Qhat = qhinv + 2 * L;
    const uint64_t* Qw = Qhat + (size_t)L * Wq;
    const uint64_t* qhb = Qw + (Wq + 1);
    const uint64_t* Qb = qhb + 2 * (size_t)L * nb;
    uint64_t y[32];
    uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    for (int i = 0; i < L; ++i) {
        y[i] = mul_shoup(x[(size_t)i * N + n], qhinv[2 * i], qhinv[2 * i + 1], mods[i].q);
        acc_mac192(w0, w1, w2, w3, y[i], fast[2 * i], fast[2 * i + 1]);
    }
    uint64_t v = w2 + (w1 >> 63);
    if (w1 == kNearHalf || force_exact) {
        uint64_t X[HE_MW_MAX + 1];
        for (int w = 0; w <= Wq; ++w) X[w] = 0;
        for (int i = 0; i < L; ++i) mw_mac(X, Qhat + (size_t)i * Wq, Wq, y[i]);
        v = 0;
        while (mw_cmp(X, Qw, Wq + 1) >= 0) {
            mw_sub(X, Qw, Wq + 1);
            ++v;
        }
        uint64_t X2[HE_MW_MAX + 1];   // centred: x > Q/2 (i.e. 2x > Q) -> x - Q
        uint64_t c = 0;
        for (int w = 0; w <= Wq; ++w) {
            X2[w] = (X[w] << 1) | c;
            c = X[w] >> 63;
        }
        if (mw_cmp(X2, Qw, Wq + 1) > 0) ++v;
    }
    for (int j = 0; j < nb; ++j) {
        const uint64_t b = mods[b_off + j].q;
        uint64_t z = 0;
        for (int i = 0; i < L; ++i) {
            const uint64_t* p = qhb + 2 * ((size_t)i * nb + j);
            z = add_mod(z, mul_shoup(y[i], p[0], p[1], b), b);
        }
        z = sub_mod(z, mul_shoup(v, Qb[2 * j], Qb[2 * j + 1], b), b);
        x[(size_t)(L + j) * N + n] = z;
    }
}

// Tensor product over the R = L + nb limbs (NTT domain): D = (a0 b0, a0 b1 + a1 b0, a1 b1);
// item blockIdx.z, A and Bv [items][2][R][N], D [items][3][R][N].
__global__ void k_tensor(const uint64_t* __restrict__ A, const uint64_t* __restrict__ Bv,
                         uint64_t* __restrict__ D, int R, int L, int b_off, int logN,
                         const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.y;
    const ModConst M = mods[r < L ? r : b_off + (r - L)];
    const size_t RN = (size_t)R * N;
    const size_t off = (size_t)r * N + n, it = blockIdx.z;
    A += it * 2 * RN;
    Bv += it * 2 * RN;
    D += it * 3 * RN;
    const uint64_t a0 = A[off], a1 = A[RN + off];
    const uint64_t b0 = to_mont(Bv[off], M), b1 = to_mont(Bv[RN + off], M);
    U128 p0{0, 0}, p1{0, 0}, p2{0, 0};
    mac128(p0, a0, b0);
    mac128(p1, a0, b1);
    mac128(p1, a1, b0);
    mac128(p2, a1, b1);
    D[off] = redc(p0, M.q, M.qinv_neg);
    D[RN + off] = redc(p1, M.q, M.qinv_neg);
    D[2 * RN + off] = redc(p2, M.q, M.qinv_neg);
}

// round(t d / Q) by multi-word arithmetic: d = sum_m y_m Mhat_m reduced mod M, centred in
// (-M/2, M/2]; |d| = A, round(t A / Q) = floor((2 t A + Q) / 2Q) by binary long division (no
// ties: Q odd, gcd(Q, t) = 1), negated for negative d; written mod each q_i to s[i N].
// Table: mhinv[R] pairs | Mhat[R][Wm] | M[Wm+1] | Q[Wm+2] | Q2[Wm+2]
__device__ void scale_round_multiword(const uint64_t* y, uint64_t* s, int n, int N, int R, int L,
                                      int Wm, uint64_t t, const ModConst* __restrict__ mods,
                                      const uint64_t* __restrict__ tab) {
    const uint64_t* Mhat = tab + 2 * R;
    const uint64_t* Mw = Mhat + (size_t)R * Wm;
    const uint64_t* Qw = Mw + (Wm + 1);
    const uint64_t* Q2w = Qw + (Wm + 2);
    const int W = Wm + 2;
    uint64_t X[HE_MW_MAX + 2];
    for (int w = 0; w < W; ++w) X[w] = 0;
    for (int m = 0; m < R; ++m) mw_mac(X, Mhat + (size_t)m * Wm, Wm, y[m]);
    while (mw_cmp(X, Mw, Wm + 1) >= 0) mw_sub(X, Mw, Wm + 1);
    // sign: d = X - M when 2X > M
    uint64_t A[HE_MW_MAX + 2];
    uint64_t c = 0;
    for (int w = 0; w < W; ++w) {
        A[w] = (w <= Wm ? (X[w] << 1) | c : c);
        c = w <= Wm ? X[w] >> 63 : 0;
    }
    uint64_t Mpad[HE_MW_MAX + 2];
    for (int w = 0; w < W; ++w) Mpad[w] = w <= Wm ? Mw[w] : 0;
    const bool neg = mw_cmp(A, Mpad, W) > 0;
    for (int w = 0; w < W; ++w) A[w] = w <= Wm ? X[w] : 0;
    if (neg) {                               // A = M - X
        uint64_t T[HE_MW_MAX + 2];
        for (int w = 0; w < W; ++w) T[w] = Mpad[w];
        mw_sub(T, A, W);
        for (int w = 0; w < W; ++w) A[w] = T[w];
    }
    uint64_t num[HE_MW_MAX + 2];             // num = 2 t A + Q
    {
        uint64_t carry = 0;
        for (int w = 0; w < W; ++w) {
            unsigned __int128 p = (unsigned __int128)A[w] * (2 * t) + carry;
            num[w] = (uint64_t)p;
            carry = (uint64_t)(p >> 64);
        }
        unsigned __int128 sum = 0;
        for (int w = 0; w < W; ++w) {
            sum += (unsigned __int128)num[w] + Qw[w];
            num[w] = (uint64_t)sum;
            sum >>= 64;
        }
    }
    int top = W - 1;                         // quotient = floor(num / 2Q)
    while (top > 0 && num[top] == 0) --top;
    uint64_t rem[HE_MW_MAX + 2], quo[HE_MW_MAX + 2];
    for (int w = 0; w < W; ++w) rem[w] = quo[w] = 0;
    for (int bit = top * 64 + 63; bit >= 0; --bit) {
        uint64_t cc = (num[bit >> 6] >> (bit & 63)) & 1u;
        for (int w = 0; w < W; ++w) {        // rem = (rem << 1) | bit
            const uint64_t nx = rem[w] >> 63;
            rem[w] = (rem[w] << 1) | cc;
            cc = nx;
        }
        if (mw_cmp(rem, Q2w, W) >= 0) {
            mw_sub(rem, Q2w, W);
            quo[bit >> 6] |= 1ull << (bit & 63);
        }
    }
    for (int i = 0; i < L; ++i) {
        const uint64_t q = mods[i].q;
        const uint64_t r = mw_mod(quo, W, q);
        s[(size_t)i * N + n] = neg ? (r ? q - r : 0) : r;
    }
}

// round(t d / Q) mod q_i for each product polynomial (coefficient form over Q u B in, over Q
// out), without multi-word integers.  With d = sum_m y_m Mhat_m - v M (M = Q B), y_m =
// [d_m Mhat_m^-1]_{m_m}:
//   t Mhat_i / Q = t B / q_i = a_i + r_i / q_i     (a_i = floor(t B / q_i), r_i = t B mod q_i)
//   t Mhat_m / Q = t Bhat_j  (m = L + j, an integer),  t M / Q = t B,
// so t d / Q = I + F with the integer I = sum_i y_i a_i + sum_j y_{L+j} t Bhat_j - v t B and
// F = sum_i y_i r_i / q_i, and round(t d / Q) = I + round(F) (no ties).  v = round(sum_m
// y_m / m_m) is unambiguous because |d| <= N Q^2 / 2 < M / 32 (prod B > 16 N Q).  I is formed
// modulo each q_k from the tables; round(F) from the 128-bit fractions phi_i of r_i / q_i,
// with the multi-word path when the fixed-point bound is inconclusive (or force_exact).
// blockIdx.y = 3 item + k; d0, d1 go to S01 [items][2][L][N], d2 to the c1 half of
// T2 [items][2][L][N] (the layout the key switch reads).
// Fast table: G[R] (hi, lo) = floor(2^128 / m_m) | phi[L] (hi, lo) | C[L][R + 1] Montgomery:
// C[k][i] = [a_i]_{q_k}, C[k][L + j] = [t Bhat_j]_{q_k}, C[k][R] = [t B]_{q_k}.
__global__ void k_scale_round(const uint64_t* __restrict__ D, uint64_t* __restrict__ S01,
                              uint64_t* __restrict__ T2, int R, int L, int Wm, int b_off,
                              uint64_t t, int logN, const ModConst* __restrict__ mods,
                              const uint64_t* __restrict__ tab, const uint64_t* __restrict__ fast,
                              int force_exact) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int it = blockIdx.y / 3, k = blockIdx.y - 3 * it;
    const uint64_t* d = D + (size_t)blockIdx.y * R * N;
    const uint64_t* mhinv = tab;
    const uint64_t* G = fast;
    const uint64_t* phi = G + 2 * R;
    const uint64_t* C = phi + 2 * L;
    uint64_t* s = k < 2 ? S01 + ((size_t)it * 2 + k) * L * N : T2 + ((size_t)it * 2 + 1) * L * N;
    uint64_t y[HE_MW_MAX * 2];
    U128 sv{0, 0};
    for (int m = 0; m < R; ++m) {
        const uint64_t q = mods[m < L ? m : b_off + (m - L)].q;
        y[m] = mul_shoup(d[(size_t)m * N + n], mhinv[2 * m], mhinv[2 * m + 1], q);
        mac128(sv, y[m], G[2 * m]);                 // y_m / m_m in units of 2^-64
        const uint64_t h = mulhi64(y[m], G[2 * m + 1]);
        sv.lo += h;
        sv.hi += sv.lo < h;
    }
    const uint64_t v = sv.hi + (sv.lo >> 63);
    uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    for (int i = 0; i < L; ++i) acc_mac192(w0, w1, w2, w3, y[i], phi[2 * i], phi[2 * i + 1]);
    if (w1 == kNearHalf || force_exact) {
        scale_round_multiword(y, s, n, N, R, L, Wm, t, mods, tab);
        return;
    }
    // round(F) = w3 2^64 + w2 + [w1 >= 2^63] (< 2^66)
    U128 f{w2 + (w1 >> 63), w3};
    f.hi += f.lo < (w1 >> 63);
    for (int kk = 0; kk < L; ++kk) {
        const ModConst M = mods[kk];
        const uint64_t* c = C + (size_t)kk * (R + 1);
        uint64_t acc = 0;
        for (int m = 0; m < R; ++m) {
            U128 p{0, 0};
            mac128(p, y[m], c[m]);
            acc = add_mod(acc, redc(p, M.q, M.qinv_neg), M.q);
        }
        U128 pv{0, 0};
        mac128(pv, v, c[R]);
        acc = sub_mod(acc, redc(pv, M.q, M.qinv_neg), M.q);
        // [round(F)]_{q_k}: f 2^-64 by REDC, then back to f by a Montgomery product with 2^128
        const uint64_t fr = to_mont(redc(f, M.q, M.qinv_neg), M);
        s[(size_t)kk * N + n] = add_mod(acc, fr, M.q);
    }
}

uint64_t h_mulmod_(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((unsigned __int128)a * b % q); }

void mw_mul_small_h(std::vector<uint64_t>& a, uint64_t m) {
    unsigned __int128 carry = 0;
    for (auto& w : a) {
        unsigned __int128 p = (unsigned __int128)w * m + carry;
        w = (uint64_t)p;
        carry = p >> 64;
    }
    if (carry) a.push_back((uint64_t)carry);
}

std::vector<uint64_t> padded(std::vector<uint64_t> v, size_t W) {
    v.resize(W, 0);
    return v;
}

// a / d (multi-word by one word): quotient into quo, remainder returned.
uint64_t mw_divmod_h(const std::vector<uint64_t>& a, uint64_t d, std::vector<uint64_t>& quo) {
    quo.assign(a.size(), 0);
    unsigned __int128 r = 0;
    for (size_t w = a.size(); w-- > 0;) {
        r = (r << 64) | a[w];
        quo[w] = (uint64_t)(r / d);
        r %= d;
    }
    return (uint64_t)r;
}

uint64_t mw_mod_h(const std::vector<uint64_t>& a, uint64_t d) {
    std::vector<uint64_t> q;
    return mw_divmod_h(a, d, q);
}

// floor(x 2^128 / d) for x < d, as (hi, lo)
void frac128_h(uint64_t x, uint64_t d, std::vector<uint64_t>& out) {
    unsigned __int128 r = (unsigned __int128)x << 64;
    out.push_back((uint64_t)(r / d));
    r = (r % d) << 64;
    out.push_back((uint64_t)(r / d));
}

}  // namespace

// Tables of the exact extension (level L) and of the scale-and-round, built once per context.
static int mult_tables(he_ctx* ctx) {
    if (ctx->d_mult_tab) return HE_OK;
    const int L = ctx->L, nb = ctx->n_b, R = L + nb, b_off = ctx->L + ctx->K + 1;
    std::vector<uint64_t> mods_r(R);
    for (int m = 0; m < R; ++m) mods_r[m] = ctx->mods[m < L ? m : b_off + (m - L)];
    std::vector<uint64_t> Q{1}, M{1};
    for (int i = 0; i < L; ++i) mw_mul_small_h(Q, ctx->mods[i]);
    for (int m = 0; m < R; ++m) mw_mul_small_h(M, mods_r[m]);
    const int Wq = (int)Q.size(), Wm = (int)M.size();
    if (Wm + 2 > HE_MW_MAX) return he_fail(ctx, HE_EINVAL, "he_multiply: modulus too large");
    std::vector<uint64_t> ext, sc;
    // extension table
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = ctx->mods[i];
        uint64_t v = 1;
        for (int k = 0; k < L; ++k)
            if (k != i) v = h_mulmod_(v, ctx->mods[k] % qi, qi);
        ShoupPair p = h_shoup(h_inv(v, qi), qi);
        ext.push_back(p.w);
        ext.push_back(p.ws);
    }
    for (int i = 0; i < L; ++i) {
        std::vector<uint64_t> qh{1};
        for (int k = 0; k < L; ++k)
            if (k != i) mw_mul_small_h(qh, ctx->mods[k]);
        qh = padded(qh, Wq);
        ext.insert(ext.end(), qh.begin(), qh.end());
    }
    {
        std::vector<uint64_t> q1 = padded(Q, Wq + 1);
        ext.insert(ext.end(), q1.begin(), q1.end());
    }
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < nb; ++j) {
            const uint64_t b = ctx->mods[b_off + j];
            uint64_t v = 1;
            for (int k = 0; k < L; ++k)
                if (k != i) v = h_mulmod_(v, ctx->mods[k] % b, b);
            ShoupPair p = h_shoup(v, b);
            ext.push_back(p.w);
            ext.push_back(p.ws);
        }
    for (int j = 0; j < nb; ++j) {
        const uint64_t b = ctx->mods[b_off + j];
        uint64_t v = 1;
        for (int k = 0; k < L; ++k) v = h_mulmod_(v, ctx->mods[k] % b, b);
        ShoupPair p = h_shoup(v, b);
        ext.push_back(p.w);
        ext.push_back(p.ws);
    }
    // scale table
    for (int m = 0; m < R; ++m) {
        const uint64_t qm = mods_r[m];
        uint64_t v = 1;
        for (int k = 0; k < R; ++k)
            if (k != m) v = h_mulmod_(v, mods_r[k] % qm, qm);
        ShoupPair p = h_shoup(h_inv(v, qm), qm);
        sc.push_back(p.w);
        sc.push_back(p.ws);
    }
    for (int m = 0; m < R; ++m) {
        std::vector<uint64_t> mh{1};
        for (int k = 0; k < R; ++k)
            if (k != m) mw_mul_small_h(mh, mods_r[k]);
        mh = padded(mh, Wm);
        sc.insert(sc.end(), mh.begin(), mh.end());
    }
    {
        std::vector<uint64_t> m1 = padded(M, Wm + 1);
        sc.insert(sc.end(), m1.begin(), m1.end());
        std::vector<uint64_t> q2 = padded(Q, Wm + 2);
        sc.insert(sc.end(), q2.begin(), q2.end());
        std::vector<uint64_t> qq = Q;
        mw_mul_small_h(qq, 2);
        qq = padded(qq, Wm + 2);
        sc.insert(sc.end(), qq.begin(), qq.end());
    }
    // fixed-point tables: psi_i = 2^128 / q_i (extension); G_m = 2^128 / m_m, phi_i =
    // 2^128 (t B mod q_i) / q_i and the Montgomery constants C[k][.] (scale)
    std::vector<uint64_t> extf, scf;
    for (int i = 0; i < L; ++i) frac128_h(1, ctx->mods[i], extf);
    std::vector<uint64_t> Bw{1}, tB;
    for (int j = 0; j < nb; ++j) mw_mul_small_h(Bw, ctx->mods[b_off + j]);
    tB = Bw;
    mw_mul_small_h(tB, ctx->prm.t);
    for (int m = 0; m < R; ++m) frac128_h(1, mods_r[m], scf);
    for (int i = 0; i < L; ++i) frac128_h(mw_mod_h(tB, ctx->mods[i]), ctx->mods[i], scf);
    std::vector<std::vector<uint64_t>> a(L), tbh(nb);
    for (int i = 0; i < L; ++i) mw_divmod_h(tB, ctx->mods[i], a[i]);
    for (int j = 0; j < nb; ++j) {
        mw_divmod_h(Bw, ctx->mods[b_off + j], tbh[j]);
        mw_mul_small_h(tbh[j], ctx->prm.t);
    }
    for (int k = 0; k < L; ++k) {
        const uint64_t qk = ctx->mods[k];
        for (int i = 0; i < L; ++i) scf.push_back(h_to_mont(mw_mod_h(a[i], qk), qk));
        for (int j = 0; j < nb; ++j) scf.push_back(h_to_mont(mw_mod_h(tbh[j], qk), qk));
        scf.push_back(h_to_mont(mw_mod_h(tB, qk), qk));
    }
    ctx->mult_ext_words = ext.size();
    ctx->mult_extf_off = ext.size() + sc.size();
    ctx->mult_scf_off = ctx->mult_extf_off + extf.size();
    ctx->mult_Wq = Wq;
    ctx->mult_Wm = Wm;
    std::vector<uint64_t> all = ext;
    all.insert(all.end(), sc.begin(), sc.end());
    all.insert(all.end(), extf.begin(), extf.end());
    all.insert(all.end(), scf.begin(), scf.end());
    if (cudaMalloc((void**)&ctx->d_mult_tab, all.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "he_multiply: table allocation failed");
    }
    HE_CHECK_CUDA(ctx, cudaMemcpy(ctx->d_mult_tab, all.data(), all.size() * 8, cudaMemcpyHostToDevice));
    return HE_OK;
}

// Products of n pairs (a[i], b[i]) into out[i], in chunks that bound the scratch.
static int multiply_items(he_ctx* ctx, const he_ct* a, const he_ct* b, int n, he_ct* out,
                          const uint64_t* rlk) {
    const int L = ctx->L, nb = ctx->n_b, R = L + nb, b_off = ctx->L + ctx->K + 1;
    const size_t N = ctx->N, ct = 2 * (size_t)L * N, ext = 2 * (size_t)R * N;
    const size_t per_item = 2 * ext + 3 * (size_t)R * N + 2 * ct + rot_scratch_per_item(ctx);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n, (size_t(3) << 30) / 8 / per_item));
    const uint64_t* ext_tab = ctx->d_mult_tab;
    const uint64_t* sc_tab = ctx->d_mult_tab + ctx->mult_ext_words;
    const uint64_t* extf_tab = ctx->d_mult_tab + ctx->mult_extf_off;
    const uint64_t* scf_tab = ctx->d_mult_tab + ctx->mult_scf_off;
    // HE_MULT_EXACT=1 takes the multi-word rounding path for every coefficient (a check of
    // that path; the results are the same either way)
    const char* fe = getenv("HE_MULT_EXACT");
    const int force_exact = fe && fe[0] == '1';
    int rc;
    for (int i0 = 0; i0 < n; i0 += chunk) {
        const int m = std::min(chunk, n - i0);
        bool same = true;
        for (int i = 0; i < m; ++i) same &= a[i0 + i].data == b[i0 + i].data;
        if ((rc = arena_reserve(ctx, (size_t)m * per_item + 16 * 32))) return rc;
        arena_reset(ctx);
        uint64_t* A = arena_take(ctx, (size_t)m * ext);
        uint64_t* Bx = same ? A : arena_take(ctx, (size_t)m * ext);
        uint64_t* D = arena_take(ctx, (size_t)m * 3 * R * N);
        uint64_t* S01 = arena_take(ctx, (size_t)m * ct);
        uint64_t* T2 = arena_take(ctx, (size_t)m * ct);
        RotBufs rb = rot_bufs_take(ctx, m);
        if (!rb.v) return he_fail(ctx, HE_ENOMEM, "he_multiply: scratch");
        for (int u = 0; u < (same ? 1 : 2); ++u) {
            const he_ct* src = u ? b : a;
            uint64_t* X = u ? Bx : A;
            for (int i = 0; i < m; ++i)
                for (int k = 0; k < 2; ++k)
                    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + (size_t)i * ext + (size_t)k * R * N,
                                                       src[i0 + i].data + (size_t)k * L * N,
                                                       (size_t)L * N * 8, cudaMemcpyDeviceToDevice,
                                                       ctx->stream));
            ntt_inverse(ctx, X, 2 * m, (size_t)R * N, L, 0);
            ++ctx->launches;
            k_extend_exact<<<dim3((unsigned)((N + 127) / 128), 2 * m), 128, 0, ctx->stream>>>(
                X, (size_t)R * N, L, nb, ctx->mult_Wq, b_off, ctx->logN, ctx->d_mod, ext_tab,
                extf_tab, force_exact);
            ntt_forward(ctx, X, 2 * m, (size_t)R * N, L, 0);
            ntt_forward(ctx, X + (size_t)L * N, 2 * m, (size_t)R * N, nb, b_off);
        }
        ++ctx->launches;
        k_tensor<<<dim3((unsigned)((N + 255) / 256), R, m), 256, 0, ctx->stream>>>(
            A, Bx, D, R, L, b_off, ctx->logN, ctx->d_mod);
        ntt_inverse(ctx, D, 3 * m, (size_t)R * N, L, 0);
        ntt_inverse(ctx, D + (size_t)L * N, 3 * m, (size_t)R * N, nb, b_off);
        ++ctx->launches;
        k_scale_round<<<dim3((unsigned)((N + 127) / 128), 3 * m), 128, 0, ctx->stream>>>(
            D, S01, T2, R, L, ctx->mult_Wm, b_off, ctx->prm.t, ctx->logN, ctx->d_mod, sc_tab, scf_tab,
            force_exact);
        ntt_forward(ctx, S01, 2 * m, (size_t)L * N, L, 0);
        ntt_forward(ctx, T2 + (size_t)L * N, m, ct, L, 0);
        // relinearise: out = (d0, d1) + KeySwitch_{s^2 -> s}(d2)
        std::vector<const uint64_t*> bs(m);
        std::vector<uint64_t*> os(m);
        for (int i = 0; i < m; ++i) {
            bs[i] = S01 + (size_t)i * ct;
            os[i] = out[i0 + i].data;
        }
        auto bp = upload_ptrs(ctx, bs);
        auto op = upload_out_ptrs(ctx, os);
        if (!bp || !op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        modup_items(ctx, T2, m, 1u, rb);
        ks_items(ctx, m, rlk, 1u, 1u, nullptr, bp, op, rb);
        for (int i = 0; i < m; ++i) out[i0 + i].domain = HE_NTT;
    }
    ctx->ops[3] += (uint64_t)n;
    return HE_OK;
}

extern "C" int he_multiply_batch(he_ctx* ctx, const he_ct* a, const he_ct* b, int n, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!a || !b || !out || n < 0) return he_fail(ctx, HE_EINVAL, "he_multiply: null argument");
    int rc;
    for (int i = 0; i < n; ++i) {
        if ((rc = check_ct(ctx, &a[i], ctx->L, HE_NTT, "he_multiply a"))) return rc;
        if ((rc = check_ct(ctx, &b[i], ctx->L, HE_NTT, "he_multiply b"))) return rc;
        if ((rc = check_ct(ctx, &out[i], ctx->L, -1, "he_multiply out"))) return rc;
    }
    if (ctx->L > 32) return he_fail(ctx, HE_EINVAL, "he_multiply: at most 32 primes");
    const uint64_t* rlk = nullptr;
    if (he_get_key(ctx, 0u, &rlk))
        return he_fail(ctx, HE_ENOKEY, "he_multiply: no relinearisation key (step HE_RELIN_KEY)");
    if ((rc = mult_tables(ctx))) return rc;
    if (n == 0) return HE_OK;
    phase_begin(ctx, HE_PHASE_MULTIPLY);
    rc = multiply_items(ctx, a, b, n, out, rlk);
    phase_end(ctx);
    if (rc) return rc;
    return he_launch_check(ctx, "he_multiply");
}

extern "C" int he_multiply(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out) {
    return he_multiply_batch(ctx, a, b, 1, out);
}
