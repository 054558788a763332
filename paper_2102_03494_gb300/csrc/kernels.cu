// kernels.cu -- element-wise and base-conversion kernels of the RNS-BFV path.
//
// Layout: a ring element is [limbs][N] uint64 residues; a ciphertext [2][limbs][N].  Grids
// put the "item" (ciphertext / output) index in blockIdx.x so that CTAs running together
// touch the same coefficient tile of shared operands (keys, plaintexts) and find it in L2.
#include <algorithm>

#include "he_internal.cuh"
#include "kernels.cuh"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

}  // namespace

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t state0, uint64_t ctr) {
    return mix64(state0 + (ctr + 1ull) * kGamma);
}

// ------------------------------------------------------------------ automorphism

// out[item][r][p] = in[item][r][perm_g(p)] for `rows` limbs per item.
// The outputs of an aligned chunk of T = 2^lt consecutive positions read one aligned chunk of
// T inputs: the top logN - lt bits of perm_src(p) depend only on those of p (an odd exponent
// times g keeps its low bits a function of its low bits, and the bit reversal exchanges low
// and high bits).  One CTA per (item, chunk, row) stages the source chunk in shared memory by
// coalesced 16-byte loads, then writes its outputs in order.  With alpha > 0 output row r goes
// to row (r / alpha) lk + r: a digit's own limbs inside the ModUp layout [dnum][lk][N].
constexpr int kAutoLog = 11;   // T = 2048 residues, 16 KiB
__global__ void __launch_bounds__(256) k_automorph(const uint64_t* __restrict__ in, size_t in_stride,
                                                   uint64_t* __restrict__ out, size_t out_stride,
                                                   int logN, uint32_t g, int alpha, int lk) {
    __shared__ __align__(16) uint64_t sm[1 << kAutoLog];
    const int lt = min(logN, kAutoLog), T = 1 << lt;
    const size_t N = (size_t)1 << logN;
    const uint32_t c0 = blockIdx.y << lt;                         // first output of the chunk
    const uint32_t s0 = perm_src(c0, g, logN) & ~(uint32_t)(T - 1);
    const uint64_t* a = in + blockIdx.x * in_stride + blockIdx.z * N + s0;
    const size_t orow = alpha ? (blockIdx.z / alpha) * (size_t)lk + blockIdx.z : blockIdx.z;
    uint64_t* b = out + blockIdx.x * out_stride + orow * N + c0;
    if ((reinterpret_cast<uintptr_t>(a) & 15) == 0) {            // T is even: whole pairs
        const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(a);
        for (int i = threadIdx.x; i < T / 2; i += blockDim.x)
            reinterpret_cast<ulonglong2*>(sm)[i] = a2[i];
    } else {
        for (int i = threadIdx.x; i < T; i += blockDim.x) sm[i] = a[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T; i += blockDim.x)
        b[i] = sm[perm_src(c0 + i, g, logN) & (T - 1)];
}

// ------------------------------------------------------------------ key switching

// ModUp.  x_coeff: [item][L][N] coefficient form of the polynomial being switched;
// x_ntt: [item][L][N] its NTT form (read at perm_g positions for the digit's own limbs);
// out: [item][dnum][L+K][N].  Rows outside digit j get the fast base conversion
//   y_l = sum_{i in digit j} [x_i (Q_j/q_i)^-1]_{q_i} [Q_j/q_i]_{m_l}  mod m_l
// (coefficient form, transformed afterwards); the digit's own rows get the NTT form.
__global__ void k_modup(const uint64_t* __restrict__ x_coeff, size_t xc_stride,
                        const uint64_t* __restrict__ x_ntt, size_t xn_stride, uint32_t g_own,
                        uint64_t* __restrict__ out, size_t out_stride, int L, int K, int alpha,
                        int logN, const ModConst* __restrict__ mods,
                        const ShoupPair* __restrict__ inv, const ShoupPair* __restrict__ cst,
                        int groups) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int j = blockIdx.z / groups;       // digit; the target limbs are split in `groups`
    const int grp = blockIdx.z - j * groups;
    const int LK = L + K;
    const int l_lo = grp * LK / groups, l_hi = (grp + 1) * LK / groups;
    const int i0 = j * alpha;
    const int i1 = min(i0 + alpha, L);
    const uint64_t* xc = x_coeff + blockIdx.x * xc_stride;
    const uint64_t* xn = x_ntt + blockIdx.x * xn_stride;
    uint64_t* o = out + blockIdx.x * out_stride + (size_t)j * LK * N;
    const int na = i1 - i0;                  // primes in this digit (<= 8)
    uint64_t y[8];                           // unrolled with constant indices: registers
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        y[k] = 0;
        if (k < na) {
            const ShoupPair w = inv[i0 + k];
            y[k] = mul_shoup(xc[(size_t)(i0 + k) * N + n], w.w, w.ws, mods[i0 + k].q);
        }
    }
    const uint32_t src = perm_src(n, g_own, logN);
    for (int l = l_lo; l < l_hi; ++l) {
        if (l >= i0 && l < i1) {
            o[(size_t)l * N + n] = xn[(size_t)l * N + src];
            continue;
        }
        const uint64_t ql = mods[l].q;
        const ShoupPair* cl = cst + (size_t)j * alpha * LK + l;
        uint64_t acc = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k < na) {
                const ShoupPair c = cl[(size_t)k * LK];
                acc = add_mod(acc, mul_shoup(y[k], c.w, c.ws, ql), ql);
            }
        }
        o[(size_t)l * N + n] = acc;
    }
}

// Inner product with a key in Montgomery form: u_k[l][p] = sum_j D_j[l][perm_g(p)] * key_j,k[l][p]
// D: [item][dnum][L+K][N]; key: [dnum][2][L+K][N]; u: [item][2][L+K][N].
__global__ void k_ks_inner(const uint64_t* __restrict__ D, size_t d_stride,
                           const uint64_t* __restrict__ key, uint64_t* __restrict__ u,
                           size_t u_stride, int LK, int dnum, int logN, uint32_t g,
                           const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.z;
    const ModConst M = mods[l];
    const uint32_t src = perm_src(n, g, logN);
    const uint64_t* d = D + blockIdx.x * d_stride + (size_t)l * N;
    const uint64_t* kb = key + (size_t)l * N + n;
    U128 a0{0, 0}, a1{0, 0};
    for (int j = 0; j < dnum; ++j) {
        uint64_t x = d[(size_t)j * LK * N + src];
        mac128r(a0, x, kb[(size_t)(2 * j) * LK * N]);
        mac128r(a1, x, kb[(size_t)(2 * j + 1) * LK * N]);
    }
    uint64_t* ub = u + blockIdx.x * u_stride + (size_t)l * N + n;
    ub[0] = redc(a0, M.q, M.qinv_neg);
    ub[(size_t)LK * N] = redc(a1, M.q, M.qinv_neg);
}

// ModDown base conversion.  u: [item][2][L+K][N] with the K special rows in coefficient form;
// v: [item][2][L][N] coefficient form, v_i = sum_k [u_{p_k} (P/p_k)^-1]_{p_k} [P/p_k]_{q_i}.
__global__ void k_moddown_conv(const uint64_t* __restrict__ u, size_t u_stride,
                               uint64_t* __restrict__ v, size_t v_stride, int L, int K,
                               int logN, const ModConst* __restrict__ mods,
                               const ShoupPair* __restrict__ inv,
                               const ShoupPair* __restrict__ cst, int groups) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int k = blockIdx.z / groups;       // polynomial 0 or 1; its limbs split in `groups`
    const int grp = blockIdx.z - k * groups;
    const int i_lo = grp * L / groups, i_hi = (grp + 1) * L / groups;
    const int LK = L + K;
    const uint64_t* ub = u + blockIdx.x * u_stride + (size_t)k * LK * N + (size_t)L * N;
    uint64_t y[8];                           // K <= 8; constant indices keep y in registers
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        y[kk] = 0;
        if (kk < K) {
            const ShoupPair w = inv[kk];
            y[kk] = mul_shoup(ub[(size_t)kk * N + n], w.w, w.ws, mods[L + kk].q);
        }
    }
    uint64_t* vb = v + blockIdx.x * v_stride + (size_t)k * L * N;
    for (int i = i_lo; i < i_hi; ++i) {
        const uint64_t qi = mods[i].q;
        uint64_t acc = 0;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            if (kk < K) {
                const ShoupPair c = cst[(size_t)kk * L + i];
                acc = add_mod(acc, mul_shoup(y[kk], c.w, c.ws, qi), qi);
            }
        }
        vb[(size_t)i * N + n] = acc;
    }
}

// Rotation result: out_k[i] = (u_k[i] - v_k[i]) P^-1 (+ c0[i][perm_g] for k = 0)
// (+ base_k[i] when base != null).  All NTT domain.  out/base/c0 addressed through pointer
// tables (one pointer per item, each a [2][L][N] ciphertext).
__global__ void k_ks_combine(const uint64_t* __restrict__ u, size_t u_stride,
                             const uint64_t* __restrict__ v, size_t v_stride,
                             const uint64_t* const* __restrict__ c0p,
                             const uint64_t* const* __restrict__ basep, uint64_t* const* outp,
                             int L, int K, int logN, uint32_t g,
                             const ModConst* __restrict__ mods,
                             const ShoupPair* __restrict__ pinv) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const int LK = L + K;
    const uint64_t q = mods[i].q;
    const ShoupPair w = pinv[i];
    const uint32_t src = perm_src(n, g, logN);
    const int it = blockIdx.x;
    const uint64_t* ub = u + it * u_stride + (size_t)i * N + n;
    const uint64_t* vb = v + it * v_stride + (size_t)i * N + n;
    uint64_t r0 = mul_shoup(sub_mod(ub[0], vb[0], q), w.w, w.ws, q);
    uint64_t r1 = mul_shoup(sub_mod(ub[(size_t)LK * N], vb[(size_t)L * N], q), w.w, w.ws, q);
    if (c0p) r0 = add_mod(r0, c0p[it][(size_t)i * N + src], q);
    if (basep) {
        const uint64_t* bb = basep[it] + (size_t)i * N + n;
        r0 = add_mod(r0, bb[0], q);
        r1 = add_mod(r1, bb[(size_t)L * N], q);
    }
    uint64_t* ob = outp[it] + (size_t)i * N + n;
    ob[0] = r0;
    ob[(size_t)L * N] = r1;
}

// REDC for x < 2q 2^64 (a sum of products plus one residue times 2^64): result in [0, q).
__device__ __forceinline__ uint64_t redc_wide(U128 x, uint64_t q, uint64_t qinv_neg) {
    const uint64_t m = x.lo * qinv_neg;
    mac128(x, m, q);
    uint64_t t = x.hi;   // < 3q
    t = t >= q ? t - q : t;
    return t >= q ? t - q : t;
}

// XP[b][k][l][n] = P * x_k[l][n] mod q_l for the ciphertext limbs (P c0, P c1 of each input).
__global__ void k_scale_p(const uint64_t* __restrict__ X, uint64_t* __restrict__ XP, int L, int logN,
                          const ModConst* __restrict__ mods, const uint64_t* __restrict__ pm) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int kl = blockIdx.z, l = kl % L;
    const ModConst M = mods[l];
    const size_t off = ((size_t)blockIdx.x * 2 * L + kl) * N + n;
    U128 p{0, 0};
    mac128(p, X[off], pm[l]);
    XP[off] = redc(p, M.q, M.qinv_neg);
}

// Extended-basis tap MAC (FFConv W1 under DensePack with hoisted rotations, one ModDown per
// channel): for coefficient n of limb l of image b,
//   acc_k[c'] = sum_tap pt[c'][tap] * x_k(tap)   over Q u P, with
//   x_0(tap) = sum_j D_j[perm_g(n)] key_j,0 + (P c0)[perm_g(n)],  x_1(tap) = sum_j D_j[perm_g(n)] key_j,1
// ((P c0, P c1) unrotated for the zero offset; P = 0 modulo the special primes).
// D: [B][DNUM][L+K][N]; XP: [B][2][L][N] (P times the inputs); pts: [r][taps][L+K][N]
// Montgomery form; A: [B][r][2][L+K][N].  One thread handles two images and two channels
// (c_lo, c_lo + 1 when c_cnt = 2), so each key and plaintext value it loads serves four
// products; the grid's x dimension walks image pairs so that CTAs sharing a key tile run
// together.  Plaintext products are summed unreduced in 128 bits and reduced every 8 taps.
template <int DNUM>
__global__ void __launch_bounds__(256)
k_ks_mac_ext(const uint64_t* __restrict__ D, const uint64_t* __restrict__ XP,
             const uint64_t* __restrict__ pts, TapTable tt, int c_lo, int c_cnt, int B,
             uint64_t* __restrict__ A, int L, int K, int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.z;
    const int b0 = blockIdx.x * 2;
    const int nb = B - b0 < 2 ? B - b0 : 2;
    const int LK = L + K;
    const ModConst M = mods[l];
    const uint64_t q = M.q, qi = M.qinv_neg;
    const bool qlimb = l < L;
    const size_t LN = (size_t)LK * N;
    const int ns = tt.n_sub > 0 ? tt.n_sub : 1;
    U128 a128[2][2][2];       // [image][channel][poly], unreduced
    uint64_t acc[2][2][2];    // reduced running sums
#pragma unroll
    for (int ib = 0; ib < 2; ++ib)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                a128[ib][c][k] = U128{0, 0};
                acc[ib][c][k] = 0;
            }
    const uint64_t* pt0 = pts + ((size_t)c_lo * tt.n) * LN + (size_t)l * N + n;
    const size_t pstride = (size_t)tt.n * LN;
    int pending = 0;
    for (int t = 0; t < tt.n; ++t) {
        const uint64_t p0 = pt0[(size_t)t * LN];
        const uint64_t p1 = c_cnt > 1 ? pt0[pstride + (size_t)t * LN] : 0;
        const uint64_t* key = tt.key[t];
        const uint64_t* Db[2];
        const uint64_t* Xb[2];
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) {
            const size_t it = (size_t)(b0 + (ib < nb ? ib : 0)) * ns + tt.sub[t];
            Db[ib] = D + it * DNUM * LN + (size_t)l * N;
            Xb[ib] = XP + it * 2 * L * N + (size_t)(qlimb ? l : 0) * N;
        }
        uint64_t x[2][2];
        if (!key) {
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                x[ib][0] = qlimb ? Xb[ib][n] : 0;
                x[ib][1] = qlimb ? Xb[ib][(size_t)L * N + n] : 0;
            }
        } else {
            const uint32_t src = perm_src(n, tt.g[t], logN);
            const uint64_t* kb = key + (size_t)l * N + n;
            uint64_t kv[DNUM][2];
#pragma unroll
            for (int j = 0; j < DNUM; ++j) {
                kv[j][0] = kb[(size_t)(2 * j) * LN];
                kv[j][1] = kb[(size_t)(2 * j + 1) * LN];
            }
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                uint64_t dv[DNUM];
#pragma unroll
                for (int j = 0; j < DNUM; ++j) dv[j] = Db[ib][(size_t)j * LN + src];
                const uint64_t c0p = qlimb ? Xb[ib][src] : 0;
                U128 s0{0, 0}, s1{0, 0};
#pragma unroll
                for (int j = 0; j < DNUM; ++j) {
                    mac128r(s0, dv[j], kv[j][0]);
                    mac128r(s1, dv[j], kv[j][1]);
                }
                s0.hi += c0p;   // + (P c0) 2^64 before the division by 2^64
                x[ib][0] = redc_wide(s0, q, qi);
                x[ib][1] = redc(s1, q, qi);
            }
        }
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                mac128r(a128[ib][0][k], x[ib][k], p0);
                mac128r(a128[ib][1][k], x[ib][k], p1);
            }
        if (++pending == 8 || t == tt.n - 1) {
            pending = 0;
#pragma unroll
            for (int ib = 0; ib < 2; ++ib)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        acc[ib][c][k] = add_mod(acc[ib][c][k], redc(a128[ib][c][k], q, qi), q);
                        a128[ib][c][k] = U128{0, 0};
                    }
        }
    }
#pragma unroll
    for (int ib = 0; ib < 2; ++ib) {
        if (ib >= nb) break;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c >= c_cnt) break;
            uint64_t* ab = A + (((size_t)(b0 + ib) * tt.r + c_lo + c) * 2) * LN + (size_t)l * N + n;
            ab[0] = acc[ib][c][0];
            ab[LN] = acc[ib][c][1];
        }
    }
}

// ------------------------------------------------------------------ MulPC / AddCC

// out[o] = (accin[o] or 0) + sum_{t < T} X[o*T + t] * P[o*T + t]   (per poly and limb)
// X entries are [2][L][N] ciphertexts, P entries [L][N] plaintexts in Montgomery form.
// The products of one output are summed in 128 bits and reduced once (T < 2^64 / q_max).
__global__ void k_mac(const uint64_t* const* __restrict__ X, const uint64_t* const* __restrict__ P,
                      int T, const uint64_t* const* __restrict__ accin, uint64_t* const* outp,
                      int L, int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const int o = blockIdx.x;
    const ModConst M = mods[i];
    const size_t off = (size_t)i * N + n;
    U128 a0{0, 0}, a1{0, 0};
    for (int t = 0; t < T; ++t) {
        const uint64_t* x = X[(size_t)o * T + t];
        uint64_t p = P[(size_t)o * T + t][off];
        mac128r(a0, x[off], p);
        mac128r(a1, x[off + (size_t)L * N], p);
    }
    uint64_t r0 = redc(a0, M.q, M.qinv_neg);
    uint64_t r1 = redc(a1, M.q, M.qinv_neg);
    if (accin && accin[o]) {
        r0 = add_mod(r0, accin[o][off], M.q);
        r1 = add_mod(r1, accin[o][off + (size_t)L * N], M.q);
    }
    outp[o][off] = r0;
    outp[o][off + (size_t)L * N] = r1;
}

// ConvPack with scalar weights (Table II): out[b][c] = sum_{c'} w[c][c'] x[b][c'], weights in
// Montgomery form per limb: wm[(c * r + c') * L + i].  x: [B][r][2][L][N] contiguous.
__global__ void k_convpack(const uint64_t* __restrict__ x, int r, int O_c,
                           const uint64_t* __restrict__ wm, uint64_t* const* outp, int L,
                           int logN, const ModConst* __restrict__ mods) {
    // one thread per (image, limb, coefficient) computes every output channel: the r input
    // residues are read from HBM once (then from L1), each output written once
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const int b = blockIdx.x;
    const ModConst M = mods[i];
    const size_t ct = (size_t)2 * L * N;
    const uint64_t* xb = x + (size_t)b * r * ct + (size_t)i * N + n;
    for (int c = 0; c < O_c; ++c) {
        U128 a0{0, 0}, a1{0, 0};
        for (int cp = 0; cp < r; ++cp) {
            const uint64_t w = wm[((size_t)c * r + cp) * L + i];
            mac128r(a0, xb[cp * ct], w);
            mac128r(a1, xb[cp * ct + (size_t)L * N], w);
        }
        uint64_t* ob = outp[(size_t)b * O_c + c] + (size_t)i * N + n;
        ob[0] = redc(a0, M.q, M.qinv_neg);
        ob[(size_t)L * N] = redc(a1, M.q, M.qinv_neg);
    }
}

// The same with R <= 8 inputs held in registers: each input residue is loaded once, then every
// output channel is formed from the registers.
template <int R>
__global__ void k_convpack_reg(const uint64_t* __restrict__ x, int O_c,
                               const uint64_t* __restrict__ wm, uint64_t* const* outp, int L,
                               int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const int b = blockIdx.x;
    const ModConst M = mods[i];
    const size_t ct = (size_t)2 * L * N;
    const uint64_t* xb = x + (size_t)b * R * ct + (size_t)i * N + n;
    uint64_t x0[R], x1[R];
#pragma unroll
    for (int cp = 0; cp < R; ++cp) {
        x0[cp] = xb[cp * ct];
        x1[cp] = xb[cp * ct + (size_t)L * N];
    }
    for (int c = 0; c < O_c; ++c) {
        U128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int cp = 0; cp < R; ++cp) {
            const uint64_t w = wm[((size_t)c * R + cp) * L + i];
            mac128r(a0, x0[cp], w);
            mac128r(a1, x1[cp], w);
        }
        uint64_t* ob = outp[(size_t)b * O_c + c] + (size_t)i * N + n;
        ob[0] = redc(a0, M.q, M.qinv_neg);
        ob[(size_t)L * N] = redc(a1, M.q, M.qinv_neg);
    }
}

// out = a + b for `rows` limbs (pointer tables, each entry rows*N contiguous)
__global__ void k_add(const uint64_t* const* ap, const uint64_t* const* bp, uint64_t* const* op,
                      int rows_per_poly, int polys, int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int row = blockIdx.z;
    const uint64_t q = mods[row % rows_per_poly].q;
    const size_t off = (size_t)row * N + n;
    op[blockIdx.x][off] = add_mod(ap[blockIdx.x][off], bp[blockIdx.x][off], q);
    (void)polys;
}

// bad |= 1 when some residue of `rows` rows (row r modulo mods[r % period]) is not below it.
__global__ void k_check_range(const uint64_t* __restrict__ x, int period, int logN,
                              const ModConst* __restrict__ mods, int* bad) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.z;
    if (x[(size_t)r * N + n] >= mods[r % period].q) atomicOr(bad, 1);
}

// Convert rows to Montgomery form in place (x -> x 2^64 mod q); row r uses mods[mod_off + r % period].
__global__ void k_to_mont(uint64_t* data, int rows, int period, int mod_off, int logN,
                          const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.z;
    uint64_t* p = data + (size_t)blockIdx.x * rows * N + (size_t)r * N + n;
    *p = to_mont(*p, mods[mod_off + r % period]);
}

// Back from Montgomery form (x -> x 2^-64 mod q) in place.
__global__ void k_from_mont(uint64_t* data, int rows, int period, int mod_off, int logN,
                            const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.z;
    uint64_t* p = data + (size_t)blockIdx.x * rows * N + (size_t)r * N + n;
    const ModConst M = mods[mod_off + r % period];
    *p = redc(U128{*p, 0}, M.q, M.qinv_neg);
}

// ------------------------------------------------------------------ rescale (mod switch)

// s[item][k][i][n] = ([last_k[n] + h]_{q_last} - h) mod q_i, coefficient form, i < L-1,
// h = (q_last - 1) / 2 added to every coefficient (rounding, not truncation).
// last: [item][2][N] coefficient form of the last limb of each polynomial.
__global__ void k_rescale_spread(const uint64_t* __restrict__ last, uint64_t* __restrict__ s,
                                 int L, int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int k = blockIdx.z;
    const uint64_t ql = mods[L - 1].q;
    const uint64_t h = (ql - 1) >> 1;
    const uint64_t r = add_mod(last[((size_t)blockIdx.x * 2 + k) * N + n], h, ql);
    uint64_t* sb = s + ((size_t)blockIdx.x * 2 + k) * (L - 1) * N + n;
    for (int i = 0; i < L - 1; ++i) {
        const uint64_t qi = mods[i].q;
        sb[(size_t)i * N] = sub_mod(r % qi, h % qi, qi);   // r - h: c~_i - r = c_i - (r - h)
    }
}

// last[item][k][n] = x[item][k][L-1][n] (the limb a modulus switch drops).
__global__ void k_gather_last(const uint64_t* const* xp, uint64_t* __restrict__ last, int L,
                              int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int k = blockIdx.z;
    last[((size_t)blockIdx.x * 2 + k) * N + n] = xp[blockIdx.x][((size_t)k * L + L - 1) * N + n];
}

// out_k[i] = (x_k[i] - s_k[i]) q_last^-1 mod q_i   (NTT domain)
__global__ void k_rescale_combine(const uint64_t* const* xp, const uint64_t* __restrict__ s,
                                  uint64_t* const* outp, int L, int logN,
                                  const ModConst* __restrict__ mods,
                                  const ShoupPair* __restrict__ qinv_row) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z % (L - 1), k = blockIdx.z / (L - 1);
    const uint64_t q = mods[i].q;
    const ShoupPair w = qinv_row[i];
    uint64_t x = xp[blockIdx.x][((size_t)k * L + i) * N + n];
    uint64_t sv = s[(((size_t)blockIdx.x * 2 + k) * (L - 1) + i) * N + n];
    uint64_t y = sub_mod(x, sv, q);
    outp[blockIdx.x][((size_t)k * (L - 1) + i) * N + n] = mul_shoup(y, w.w, w.ws, q);
}

// ------------------------------------------------------------------ encoder

// Slot values (int64, taken mod t) -> NTT-order buffer mod t: buf[item][slot_pos[s]] = v[s].
__global__ void k_slots_to_ntt(const int64_t* __restrict__ v, uint64_t* __restrict__ buf,
                               const int32_t* __restrict__ slot_pos, int logN, uint64_t t) {
    const int N = 1 << logN;
    const int s = blockIdx.y * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int64_t x = v[(size_t)blockIdx.x * N + s];
    int64_t m = x % (int64_t)t;
    if (m < 0) m += (int64_t)t;
    buf[(size_t)blockIdx.x * N + slot_pos[s]] = (uint64_t)m;
}

// NTT-order buffer mod t -> slot values: v[item][s] = buf[item][slot_pos[s]].
__global__ void k_ntt_to_slots(const uint64_t* __restrict__ buf, int64_t* __restrict__ v,
                               const int32_t* __restrict__ slot_pos, int logN) {
    const int N = 1 << logN;
    const int s = blockIdx.y * blockDim.x + threadIdx.x;
    if (s >= N) return;
    v[(size_t)blockIdx.x * N + s] = (int64_t)buf[(size_t)blockIdx.x * N + slot_pos[s]];
}

// m (coefficients mod t) -> centred lift mod q_i for L limbs; Montgomery form if mont != 0.
__global__ void k_lift(const uint64_t* __restrict__ m, uint64_t* __restrict__ out, int L,
                       int logN, uint64_t t, int mont, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const uint64_t x = m[(size_t)blockIdx.x * N + n];
    uint64_t* o = out + (size_t)blockIdx.x * L * N + n;
    const bool neg = x > (t - 1) / 2;
    for (int i = 0; i < L; ++i) {
        const ModConst M = mods[i];
        uint64_t r;
        if (t <= M.q) r = neg ? M.q - (t - x) : x;          // x, t - x < q: no reduction
        else r = neg ? (M.q - ((t - x) % M.q)) % M.q : x % M.q;
        o[(size_t)i * N] = mont ? to_mont(r, M) : r;
    }
}

// ------------------------------------------------------------------ client side

// Signed coefficients -> residues for `rows` moduli starting at mod_off: out[r][n].
__global__ void k_from_signed(const int64_t* __restrict__ c, uint64_t* __restrict__ out,
                              int rows, int mod_off, int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int64_t x = c[n];
    const int r = blockIdx.z;
    const uint64_t q = mods[mod_off + r].q;
    uint64_t v;
    if (x >= 0) v = (uint64_t)x % q;
    else {
        uint64_t m = ((uint64_t)(-(x + 1)) + 1u) % q;
        v = m ? q - m : 0;
    }
    out[(size_t)r * N + n] = v;
    (void)rows;
}

// Uniform residues: out[r][n] for limb index (limb0 + r) of the generator's counter space.
__global__ void k_uniform(uint64_t state0, uint64_t* __restrict__ out, int limb0, int mod_off,
                          int logN, const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int r = blockIdx.z;
    const uint64_t q = mods[mod_off + r].q;
    const uint64_t ctr = 2ull * ((uint64_t)(limb0 + r) * N + n);
    const uint64_t hi = draw(state0, ctr), lo = draw(state0, ctr + 1);
    const uint64_t a_lo = hi * q, a_hi = __umul64hi(hi, q);
    const uint64_t b_hi = __umul64hi(lo, q);
    const uint64_t mid = a_lo + b_hi;
    out[(size_t)r * N + n] = a_hi + (mid < a_lo ? 1u : 0u);
}

// Discrete Gaussian coefficients (int64) by the cumulative table T[0..19].
__global__ void k_gaussian(uint64_t state0, int64_t* __restrict__ out, int logN,
                           const uint64_t* __restrict__ cdt) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const uint64_t u = draw(state0, (uint64_t)n);
    const uint64_t x = u >> 1;
    int64_t mag = 0;
    for (int m = 0; m < 20; ++m) mag += (x >= cdt[m]) ? 1 : 0;
    out[n] = (u & 1ull) ? -mag : mag;
}

// Ternary coefficients: v = floor(3u / 2^64) in {0, 1, 2} -> {0, +1, -1}.
__global__ void k_ternary(uint64_t state0, int64_t* __restrict__ out, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const uint64_t v = __umul64hi(draw(state0, (uint64_t)n), 3ull);
    out[n] = v == 2 ? -1 : (int64_t)v;
}

// Fresh ciphertext, coefficient form: c0 = e + Delta_i m - as_i, where as holds a*s.
__global__ void k_enc_c0(const int64_t* __restrict__ e, const uint64_t* __restrict__ m,
                         const uint64_t* __restrict__ as, const ShoupPair* __restrict__ delta,
                         uint64_t* __restrict__ c0, int L, int logN,
                         const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const uint64_t q = mods[i].q;
    const int64_t x = e[n];
    uint64_t ev = x >= 0 ? (uint64_t)x % q : (q - ((uint64_t)(-x) % q)) % q;
    uint64_t dm = mul_shoup(m[n], delta[i].w, delta[i].ws, q);
    c0[(size_t)i * N + n] = sub_mod(add_mod(ev, dm, q), as[(size_t)i * N + n], q);
    (void)L;
}

// x = c0 + c1 * s (NTT domain, s in Montgomery form), rows limbs.
__global__ void k_dec_phase(const uint64_t* __restrict__ ct, const uint64_t* __restrict__ s_m,
                            uint64_t* __restrict__ x, int rows, int logN,
                            const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const ModConst M = mods[i];
    const size_t off = (size_t)i * N + n;
    U128 p{0, 0};
    mac128(p, ct[off + (size_t)rows * N], s_m[off]);
    x[off] = add_mod(ct[off], redc(p, M.q, M.qinv_neg), M.q);
}

// x <- x * s (NTT domain, s in Montgomery form), rows limbs.
__global__ void k_mul_mont(uint64_t* __restrict__ x, const uint64_t* __restrict__ s_m, int logN,
                           const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.z;
    const ModConst M = mods[i];
    const size_t off = (size_t)i * N + n;
    U128 p{0, 0};
    mac128(p, x[off], s_m[off]);
    x[off] = redc(p, M.q, M.qinv_neg);
}

// Galois key digit: b_l = e_l - a_l s_l + [l in digit] (P mod q_l) s(X^g)_l, NTT domain over
// Q u P (s in Montgomery form; pmodq in Montgomery form).
__global__ void k_keygen_b(const uint64_t* __restrict__ a, const uint64_t* __restrict__ s_m,
                           const uint64_t* __restrict__ e, const uint64_t* __restrict__ sg,
                           uint64_t* __restrict__ b, int i0, int i1, int logN,
                           const ModConst* __restrict__ mods, const uint64_t* __restrict__ pmodq) {
    const int N = 1 << logN;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.z;
    const ModConst M = mods[l];
    const size_t off = (size_t)l * N + n;
    U128 p{0, 0};
    mac128(p, a[off], s_m[off]);
    uint64_t v = sub_mod(e[off], redc(p, M.q, M.qinv_neg), M.q);
    if (l >= i0 && l < i1) {
        U128 g{0, 0};
        mac128(g, sg[off], pmodq[l]);
        v = add_mod(v, redc(g, M.q, M.qinv_neg), M.q);
    }
    b[off] = v;
}

// Exact BFV decryption rounding, one coefficient per thread:
//   t x / Q = sum_i y_i t / q_i - v t with y_i = [x_i (Q/q_i)^-1]_{q_i};
//   write y_i t = a_i q_i + b_i; then m = (sum_i a_i + round(sum_i b_i (Q/q_i) / Q)) mod t,
// the rounding decided exactly on multi-word integers.
// cst layout: qhat_inv[L] (ShoupPair as 2 u64) | Qhat[L][W] | Q[W]
__global__ void k_dec_round(const uint64_t* __restrict__ x, uint64_t* __restrict__ m, int L,
                            int W, int logN, uint64_t t, const ModConst* __restrict__ mods,
                            const uint64_t* __restrict__ cst) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const uint64_t* qhinv = cst;
    const uint64_t* qhat = cst + 2 * L;
    const uint64_t* Qw = qhat + (size_t)L * W;
    uint64_t R[HE_DEC_MAX_WORDS + 1];
    for (int w = 0; w <= W; ++w) R[w] = 0;
    uint64_t asum = 0;
    for (int i = 0; i < L; ++i) {
        const uint64_t q = mods[i].q;
        uint64_t y = mul_shoup(x[(size_t)i * N + n], qhinv[2 * i], qhinv[2 * i + 1], q);
        unsigned __int128 yt = (unsigned __int128)y * t;
        uint64_t a = (uint64_t)(yt / q);
        uint64_t b = (uint64_t)(yt % q);
        asum = (asum + a % t) % t;
        // R += b * Qhat_i
        uint64_t carry = 0;
        for (int w = 0; w < W; ++w) {
            unsigned __int128 p = (unsigned __int128)b * qhat[(size_t)i * W + w] + R[w] + carry;
            R[w] = (uint64_t)p;
            carry = (uint64_t)(p >> 64);
        }
        R[W] += carry;
    }
    // 2R
    uint64_t R2[HE_DEC_MAX_WORDS + 2];
    uint64_t c = 0;
    for (int w = 0; w <= W; ++w) {
        R2[w] = (R[w] << 1) | c;
        c = R[w] >> 63;
    }
    R2[W + 1] = c;
    // smallest k with 2R < (2k+1) Q
    uint64_t T[HE_DEC_MAX_WORDS + 2];
    for (int w = 0; w < W; ++w) T[w] = Qw[w];
    T[W] = 0;
    T[W + 1] = 0;
    uint64_t k = 0;
    for (int iter = 0; iter <= L + 1; ++iter) {
        // compare R2 >= T
        int ge = 1;
        for (int w = W + 1; w >= 0; --w) {
            if (R2[w] != T[w]) {
                ge = R2[w] > T[w];
                break;
            }
        }
        if (!ge) break;
        ++k;
        // T += 2Q
        uint64_t cy = 0;
        for (int w = 0; w <= W + 1; ++w) {
            uint64_t q2 = w < W ? (Qw[w] << 1) | (w > 0 ? Qw[w - 1] >> 63 : 0)
                                : (w == W ? Qw[W - 1] >> 63 : 0);
            unsigned __int128 s = (unsigned __int128)T[w] + q2 + cy;
            T[w] = (uint64_t)s;
            cy = (uint64_t)(s >> 64);
        }
    }
    m[n] = (asum + k % t) % t;
}

// ------------------------------------------------------------------ launch helpers

static inline dim3 grid_nx(int items, int N, int z) {
    return dim3(items, (N + 255) / 256, z);
}

void launch_automorph(he_ctx* c, const uint64_t* in, size_t in_stride, uint64_t* out,
                      size_t out_stride, int items, int rows, uint32_t g, int alpha, int lk) {
    if (items <= 0 || rows <= 0) return;
    ++c->launches;
    const int lt = std::min(c->logN, kAutoLog);
    k_automorph<<<dim3(items, c->N >> lt, rows), 256, 0, c->stream>>>(
        in, in_stride, out, out_stride, c->logN, g, alpha, lk);
}

void launch_modup(he_ctx* c, const uint64_t* x_coeff, size_t xc_stride, const uint64_t* x_ntt,
                  size_t xn_stride, uint32_t g_own, uint64_t* out, size_t out_stride, int items) {
    ++c->launches;
    const int g = c->limb_groups > 0 ? c->limb_groups : 1;
    k_modup<<<grid_nx(items, c->N, c->dnum * g), 256, 0, c->stream>>>(
        x_coeff, xc_stride, x_ntt, xn_stride, g_own, out, out_stride, c->L, c->K, c->alpha,
        c->logN, c->d_mod, c->d_modup_inv, c->d_modup_c, g);
}

void launch_ks_inner(he_ctx* c, const uint64_t* D, size_t d_stride, const uint64_t* key,
                     uint64_t* u, size_t u_stride, int items, uint32_t g) {
    ++c->launches;
    k_ks_inner<<<grid_nx(items, c->N, c->L + c->K), 256, 0, c->stream>>>(
        D, d_stride, key, u, u_stride, c->L + c->K, c->dnum, c->logN, g, c->d_mod);
}

void launch_moddown_conv(he_ctx* c, const uint64_t* u, size_t u_stride, uint64_t* v,
                         size_t v_stride, int items) {
    ++c->launches;
    const int g = c->limb_groups > 0 ? c->limb_groups : 1;
    k_moddown_conv<<<grid_nx(items, c->N, 2 * g), 256, 0, c->stream>>>(
        u, u_stride, v, v_stride, c->L, c->K, c->logN, c->d_mod, c->d_md_inv, c->d_md_c, g);
}

void launch_ks_combine(he_ctx* c, const uint64_t* u, size_t u_stride, const uint64_t* v,
                       size_t v_stride, const uint64_t* const* c0p, const uint64_t* const* basep,
                       uint64_t* const* outp, int items, uint32_t g) {
    ++c->launches;
    k_ks_combine<<<grid_nx(items, c->N, c->L), 256, 0, c->stream>>>(
        u, u_stride, v, v_stride, c0p, basep, outp, c->L, c->K, c->logN, g, c->d_mod,
        c->d_md_pinv);
}

void launch_scale_p(he_ctx* c, const uint64_t* X, uint64_t* XP, int B) {
    ++c->launches;
    k_scale_p<<<grid_nx(B, c->N, 2 * c->L), 256, 0, c->stream>>>(X, XP, c->L, c->logN, c->d_mod,
                                                                 c->d_pmodq);
}

void launch_ks_mac_ext(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                       const TapTable& tt_in, uint64_t* A, int B) {
    TapTable tt = tt_in;
    if (tt.n_sub < 1) tt.n_sub = 1;   // one input ciphertext per image
    if (tapmac_bulk_supported(c)) {   // operands staged by bulk copies (tapmac.cu)
        launch_ks_mac_ext_bulk(c, D, XP, pts, tt, A, B);
        return;
    }
    const dim3 grid((B + 1) / 2, (c->N + 255) / 256, c->L + c->K);
    for (int c_lo = 0; c_lo < tt.r; c_lo += 2) {
        ++c->launches;
        const int cnt = tt.r - c_lo < 2 ? tt.r - c_lo : 2;
#define HE_KS_MAC(DN)                                                                         \
    k_ks_mac_ext<DN><<<grid, 256, 0, c->stream>>>(D, XP, pts, tt, c_lo, cnt, B, A, c->L, c->K,  \
                                                  c->logN, c->d_mod)
        switch (c->dnum) {
            case 1: HE_KS_MAC(1); break;
            case 2: HE_KS_MAC(2); break;
            case 3: HE_KS_MAC(3); break;
            case 4: HE_KS_MAC(4); break;
            case 5: HE_KS_MAC(5); break;
            case 6: HE_KS_MAC(6); break;
            case 7: HE_KS_MAC(7); break;
            default: HE_KS_MAC(8); break;
        }
#undef HE_KS_MAC
    }
}

void launch_mac(he_ctx* c, const uint64_t* const* X, const uint64_t* const* P, int T,
                const uint64_t* const* accin, uint64_t* const* outp, int n_out, int L) {
    ++c->launches;
    k_mac<<<grid_nx(n_out, c->N, L), 256, 0, c->stream>>>(X, P, T, accin, outp, L, c->logN,
                                                          c->d_mod);
}

void launch_convpack(he_ctx* c, const uint64_t* x, int B, int r, int O_c, const uint64_t* wm,
                     uint64_t* const* outp, int L) {
    ++c->launches;
    const dim3 grid = grid_nx(B, c->N, L);
#define HE_CONVPACK_REG(R)                                                                  \
    k_convpack_reg<R><<<grid, 256, 0, c->stream>>>(x, O_c, wm, outp, L, c->logN, c->d_mod)
    switch (r) {
        case 1: HE_CONVPACK_REG(1); break;
        case 2: HE_CONVPACK_REG(2); break;
        case 3: HE_CONVPACK_REG(3); break;
        case 4: HE_CONVPACK_REG(4); break;
        case 5: HE_CONVPACK_REG(5); break;
        case 6: HE_CONVPACK_REG(6); break;
        case 7: HE_CONVPACK_REG(7); break;
        case 8: HE_CONVPACK_REG(8); break;
        default:
            k_convpack<<<grid, 256, 0, c->stream>>>(x, r, O_c, wm, outp, L, c->logN, c->d_mod);
    }
#undef HE_CONVPACK_REG
}

void launch_add(he_ctx* c, const uint64_t* const* a, const uint64_t* const* b,
                uint64_t* const* o, int items, int L) {
    ++c->launches;
    k_add<<<grid_nx(items, c->N, 2 * L), 256, 0, c->stream>>>(a, b, o, L, 2, c->logN, c->d_mod);
}

void launch_add_rows(he_ctx* c, const uint64_t* const* a, const uint64_t* const* b,
                     uint64_t* const* o, int items, int rows_per_poly) {
    ++c->launches;
    k_add<<<grid_nx(items, c->N, 2 * rows_per_poly), 256, 0, c->stream>>>(a, b, o, rows_per_poly, 2,
                                                                          c->logN, c->d_mod);
}

void launch_check_range(he_ctx* c, const uint64_t* data, int rows, int period, int* bad) {
    ++c->launches;
    k_check_range<<<grid_nx(1, c->N, rows), 256, 0, c->stream>>>(data, period, c->logN, c->d_mod,
                                                                 bad);
}

void launch_to_mont(he_ctx* c, uint64_t* data, int items, int rows, int period, int mod_off) {
    ++c->launches;
    k_to_mont<<<grid_nx(items, c->N, rows), 256, 0, c->stream>>>(data, rows, period, mod_off,
                                                                 c->logN, c->d_mod);
}

void launch_from_mont(he_ctx* c, uint64_t* data, int items, int rows, int period, int mod_off) {
    ++c->launches;
    k_from_mont<<<grid_nx(items, c->N, rows), 256, 0, c->stream>>>(data, rows, period, mod_off,
                                                                   c->logN, c->d_mod);
}

void launch_rescale_spread(he_ctx* c, const uint64_t* last, uint64_t* s, int items, int L) {
    ++c->launches;
    k_rescale_spread<<<grid_nx(items, c->N, 2), 256, 0, c->stream>>>(last, s, L, c->logN,
                                                                     c->d_mod);
}

void launch_rescale_combine(he_ctx* c, const uint64_t* const* xp, const uint64_t* s,
                            uint64_t* const* outp, int items, int L) {
    ++c->launches;
    k_rescale_combine<<<grid_nx(items, c->N, 2 * (L - 1)), 256, 0, c->stream>>>(
        xp, s, outp, L, c->logN, c->d_mod, c->d_rs_inv + (size_t)(L - 1) * c->L);
}

void launch_slots_to_ntt(he_ctx* c, const int64_t* v, uint64_t* buf, int items) {
    ++c->launches;
    k_slots_to_ntt<<<grid_nx(items, c->N, 1), 256, 0, c->stream>>>(v, buf, c->d_slot_pos,
                                                                    c->logN, c->prm.t);
}

void launch_ntt_to_slots(he_ctx* c, const uint64_t* buf, int64_t* v, int items) {
    ++c->launches;
    k_ntt_to_slots<<<grid_nx(items, c->N, 1), 256, 0, c->stream>>>(buf, v, c->d_slot_pos,
                                                                    c->logN);
}

void launch_lift(he_ctx* c, const uint64_t* m, uint64_t* out, int items, int L, int mont) {
    ++c->launches;
    k_lift<<<grid_nx(items, c->N, 1), 256, 0, c->stream>>>(m, out, L, c->logN, c->prm.t, mont,
                                                           c->d_mod);
}

void launch_from_signed(he_ctx* c, const int64_t* v, uint64_t* out, int rows, int mod_off) {
    ++c->launches;
    k_from_signed<<<grid_nx(1, c->N, rows), 256, 0, c->stream>>>(v, out, rows, mod_off, c->logN,
                                                                 c->d_mod);
}

void launch_uniform(he_ctx* c, uint64_t state0, uint64_t* out, int rows, int limb0, int mod_off) {
    ++c->launches;
    k_uniform<<<grid_nx(1, c->N, rows), 256, 0, c->stream>>>(state0, out, limb0, mod_off,
                                                             c->logN, c->d_mod);
}

void launch_gaussian(he_ctx* c, uint64_t state0, int64_t* out) {
    ++c->launches;
    k_gaussian<<<grid_nx(1, c->N, 1), 256, 0, c->stream>>>(state0, out, c->logN, c->d_cdt);
}

void launch_ternary(he_ctx* c, uint64_t state0, int64_t* out) {
    ++c->launches;
    k_ternary<<<grid_nx(1, c->N, 1), 256, 0, c->stream>>>(state0, out, c->logN);
}

void launch_enc_c0(he_ctx* c, const int64_t* e, const uint64_t* m, const uint64_t* as,
                   const ShoupPair* delta, uint64_t* c0) {
    ++c->launches;
    k_enc_c0<<<grid_nx(1, c->N, c->L), 256, 0, c->stream>>>(e, m, as, delta, c0, c->L, c->logN,
                                                            c->d_mod);
}

void launch_dec_phase(he_ctx* c, const uint64_t* ct, const uint64_t* s_m, uint64_t* x, int rows) {
    ++c->launches;
    k_dec_phase<<<grid_nx(1, c->N, rows), 256, 0, c->stream>>>(ct, s_m, x, rows, c->logN,
                                                               c->d_mod);
}

void launch_dec_round(he_ctx* c, const uint64_t* x, uint64_t* m, int L, int W,
                      const uint64_t* cst) {
    ++c->launches;
    k_dec_round<<<(c->N + 127) / 128, 128, 0, c->stream>>>(x, m, L, W, c->logN, c->prm.t,
                                                           c->d_mod, cst);
}

void launch_dec_phase_mul(he_ctx* c, uint64_t* x, const uint64_t* s_m, int rows) {
    ++c->launches;
    k_mul_mont<<<grid_nx(1, c->N, rows), 256, 0, c->stream>>>(x, s_m, c->logN, c->d_mod);
}

void launch_keygen_b(he_ctx* c, const uint64_t* a, const uint64_t* s_m, const uint64_t* e,
                     const uint64_t* sg, uint64_t* b, int i0, int i1) {
    ++c->launches;
    k_keygen_b<<<grid_nx(1, c->N, c->L + c->K), 256, 0, c->stream>>>(a, s_m, e, sg, b, i0, i1,
                                                                     c->logN, c->d_mod, c->d_pmodq);
}

void launch_gather_last(he_ctx* c, const uint64_t* const* xp, uint64_t* last, int items, int L) {
    ++c->launches;
    k_gather_last<<<grid_nx(items, c->N, 2), 256, 0, c->stream>>>(xp, last, L, c->logN);
}
