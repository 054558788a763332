// tapmac.cu -- the extended-basis tap MAC with its operands staged by bulk asynchronous copies.
//
// Same arithmetic as k_ks_mac_ext (kernels.cu): for coefficient n of limb l of image b,
//   acc_k[c'] = sum_tap pt[c'][tap] * x_k(tap)   over Q u P,
//   x_0(tap) = sum_j D_j[perm_g(n)] key_j,0 + (P c0)[perm_g(n)],  x_1(tap) = sum_j D_j[perm_g(n)] key_j,1.
// A CTA owns an aligned tile of 128 or 256 coefficients of one limb for two images.  For every
// tap the operands the tile needs are contiguous rows of the tile's size: the 2 dnum key rows
// and the channel plaintext rows at the tile, and -- because the NTT-domain automorphism maps
// every aligned block of 2^k positions onto an aligned block of 2^k positions (the bits of p
// above bit k only feed the bits of perm(p) above bit k) -- the ModUp digit rows of the one
// aligned block that holds perm_g of the tile.  (P c0)[perm_g(n)] is one word per image and
// tap, read straight from global memory.
//
// Warp-specialised pipeline: the CTA's last warp only stages taps, with cp.async.bulk, into
// three shared-memory stages; stage s is "full" when its copied bytes have landed (an
// mbarrier with a transaction count) and "empty" when every compute warp has arrived on a
// second mbarrier after its last read of it.  The compute warps (one coefficient per thread)
// never meet at a block barrier inside the tap loop, so no warp waits for the copy issue.
// Every wait is bounded: on expiry the kernel sets a bit in the context's device error word,
// waits (again bounded) for its own copies and returns.
#include "eval.cuh"
#include "he_internal.cuh"
#include "kernels.cuh"

namespace {

// Coefficients per CTA (one per thread): 128 or 256.  Without autotuning (he_autotune) the
// tile is 128 when the key has four or more digits (large stages, four CTAs per SM), else 256.
constexpr int kMaxTile = 256;
int default_tile(int dnum) { return dnum >= 4 ? 128 : 256; }
constexpr uint32_t kWaitSpins = 1u << 20;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t polls = kWaitSpins) {
    for (uint32_t i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}


__device__ __forceinline__ uint64_t redc_w(U128 x, uint64_t q, uint64_t qinv_neg) {
    const uint64_t m = x.lo * qinv_neg;   // x < 2q 2^64: (x + m q) / 2^64 < 3q
    mac128(x, m, q);
    uint64_t t = x.hi;
    t = t >= q ? t - q : t;
    return t >= q ? t - q : t;
}

// x mod q for an unreduced sum x < 64 q^2 (q < 2^60): the high word drops below q by at most
// three subtractions of q 2^64 (a multiple of q), then REDC; the tap sums are kept in the
// Montgomery domain of the plaintexts, so REDC returns the plain residue.
__device__ __forceinline__ uint64_t reduce_sum(U128 x, uint64_t q, uint64_t qinv_neg) {
    while (x.hi >= q) x.hi -= q;
    return redc(x, q, qinv_neg);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

constexpr int kStages = 3;

// Shared-memory stage (uint64 words): keys [DNUM][2][T] | pts [2][T] | digits [2 img][DNUM][T].
// A key-less tap (the centre, no rotation) stages the rows P x [2 img][2 poly] in the digit
// area instead.
template <int DNUM, int TILE>
struct Stage {
    static constexpr int T = TILE;
    static constexpr int KEYS = 0;
    static constexpr int PTS = DNUM * 2 * T;
    static constexpr int DIG = PTS + 2 * T;
    static constexpr int XP = DIG;
    static constexpr int WORDS = DIG + (2 * DNUM > 4 ? 2 * DNUM : 4) * T;
};

// The producer warp stages tap t into stage buffer `st`, completing on `bar`.
template <int DNUM, int TILE>
__device__ __forceinline__ void issue_tap(uint64_t* st, uint64_t* bar, int t, const TapTable& tt,
                                         const uint64_t* __restrict__ D,
                                         const uint64_t* __restrict__ XPg,
                                         const uint64_t* __restrict__ pts, int c_lo, int c_cnt,
                                         int b0, int nb, int l, int L, int n0, size_t LN, int N,
                                         int logN) {
    using S = Stage<DNUM, TILE>;
    constexpr int kTile = S::T;
    const int lane = threadIdx.x & 31;
    const uint64_t* key = tt.key[t];
    const bool qlimb = l < L;
    const uint32_t row = kTile * 8;
    const int src0 = key ? (int)(perm_src((uint32_t)n0, tt.g[t], logN) & ~(uint32_t)(kTile - 1)) : n0;
    // copy list: index -> (dst, src)
    const int nkeys = key ? 2 * DNUM : 0;
    const int npts = c_cnt;
    const int ndig = key ? nb * DNUM : 0;
    const int nxp = (qlimb && !key) ? 2 * nb : 0;
    const int total = nkeys + npts + ndig + nxp;
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)total * row);
    __syncwarp();
    for (int i = lane; i < total; i += 32) {
        uint64_t* dst;
        const uint64_t* src;
        if (i < nkeys) {
            dst = st + S::KEYS + i * kTile;                          // i = 2 j + k
            src = key + (size_t)i * LN + (size_t)l * N + n0;
        } else if (i < nkeys + npts) {
            const int c = i - nkeys;
            dst = st + S::PTS + c * kTile;
            src = pts + ((size_t)(c_lo + c) * tt.n + t) * LN + (size_t)l * N + n0;
        } else if (i < nkeys + npts + ndig) {
            const int q = i - nkeys - npts, ib = q / DNUM, j = q - ib * DNUM;
            const size_t it = (size_t)(b0 + ib) * tt.n_sub + tt.sub[t];
            dst = st + S::DIG + (ib * DNUM + j) * kTile;
            src = D + (it * DNUM + j) * LN + (size_t)l * N + src0;
        } else {
            const int q = i - nkeys - npts - ndig, ib = q >> 1, k = q & 1;
            const size_t it = (size_t)(b0 + ib) * tt.n_sub + tt.sub[t];
            dst = st + S::XP + (ib * 2 + k) * kTile;
            src = XPg + (it * 2 + k) * L * N + (size_t)l * N + n0;
        }
        bulk_copy(dst, src, row, bar);
    }
}

// CTAs per SM the register budget is sized for: at 128-coefficient tiles with up to four key
// digits the three stages take 54 KB, so four CTAs (4 x 5 warps) fit; 94 registers a thread.
constexpr int min_ctas(int dnum, int tile, int arith) {
    return tile == 128 && dnum <= 4 ? (arith ? 3 : 4) : 1;
}

// Compute warps, carry-chain arithmetic: every 64 x 64-bit product is added into a 128-bit
// sum by mac128; each tap's key inner product is reduced by Montgomery (REDC, 2^-64).
template <int DNUM, int TILE>
__device__ __forceinline__ bool compute_chain(const uint64_t* __restrict__ smem, uint64_t* full, uint64_t* empty,
                                   const uint64_t* __restrict__ XPg, const TapTable& tt, int c_lo,
                                   int c_cnt, uint64_t* __restrict__ A, int b0, int nb, int l, int L,
                                   int n0, size_t LN, size_t LNq, int N, int logN, const ModConst& M,
                                   uint32_t report_polls) {
    using S = Stage<DNUM, TILE>;
    constexpr int kTile = S::T;
    const int tid = threadIdx.x;
    const bool qlimb = l < L;
    bool ok = true;
    const uint64_t q = M.q, qi = M.qinv_neg;
    const int n = n0 + tid;
    // unreduced sums of at most HE_MAX_TAPS products below q^2 each: < 64 q^2 < 2^126
    U128 a128[2][2][2];
#pragma unroll
    for (int ib = 0; ib < 2; ++ib)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 2; ++k) a128[ib][c][k] = U128{0, 0};
    for (int t = 0; t < tt.n; ++t) {
        const int s = t % kStages;
        const uint64_t* st = smem + s * S::WORDS;
        // a wait longer than report_polls is reported (error bit) and then goes on with
        // the full bound, so the warp stays in step with the producer's stages
        if (!mbar_wait(&full[s], (uint32_t)(t / kStages) & 1u, report_polls)) {
            ok = false;
            mbar_wait(&full[s], (uint32_t)(t / kStages) & 1u);
        }
        uint64_t x[2][2];
        if (!tt.key[t]) {
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                x[ib][0] = (qlimb && ib < nb) ? st[S::XP + (ib * 2) * kTile + tid] : 0;
                x[ib][1] = (qlimb && ib < nb) ? st[S::XP + (ib * 2 + 1) * kTile + tid] : 0;
            }
        } else {
            const uint32_t pn = perm_src((uint32_t)n, tt.g[t], logN);
            const int loc = (int)(pn & (kTile - 1));
            uint64_t xp[2] = {0, 0};                  // (P c0)[perm_g(n)] of each image
            if (qlimb) {
#pragma unroll
                for (int ib = 0; ib < 2; ++ib)
                    if (ib < nb)
                        xp[ib] = __ldg(XPg + ((size_t)(b0 + ib) * tt.n_sub + tt.sub[t]) * 2 * LNq +
                                       (size_t)l * N + pn);
            }
            uint64_t kv[DNUM][2];
#pragma unroll
            for (int j = 0; j < DNUM; ++j) {
                kv[j][0] = st[S::KEYS + (2 * j) * kTile + tid];
                kv[j][1] = st[S::KEYS + (2 * j + 1) * kTile + tid];
            }
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                if (ib >= nb) {
                    x[ib][0] = x[ib][1] = 0;
                    continue;
                }
                U128 s0{0, 0}, s1{0, 0};
#pragma unroll
                for (int j = 0; j < DNUM; ++j) {
                    const uint64_t d = st[S::DIG + (ib * DNUM + j) * kTile + loc];
                    mac128r(s0, d, kv[j][0]);
                    mac128r(s1, d, kv[j][1]);
                }
                s0.hi += xp[ib];                      // + (P c0) 2^64 (zero on P limbs)
                x[ib][0] = redc_w(s0, q, qi);
                x[ib][1] = redc(s1, q, qi);
            }
        }
        const uint64_t p0 = st[S::PTS + tid];
        const uint64_t p1 = c_cnt > 1 ? st[S::PTS + kTile + tid] : 0;
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);   // this warp's last read of stage s
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int k = 0; k < 2; ++k) mac128r(a128[ib][0][k], x[ib][k], p0);
        if (c_cnt > 1) {                 // uniform over the launch: one channel skips this
#pragma unroll
            for (int ib = 0; ib < 2; ++ib)
#pragma unroll
                for (int k = 0; k < 2; ++k) mac128r(a128[ib][1][k], x[ib][k], p1);
        }
    }
    if (ok) {
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) {
            if (ib >= nb) break;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c >= c_cnt) break;
                uint64_t* ab = A + (((size_t)(b0 + ib) * tt.r + c_lo + c) * 2) * LN + (size_t)l * N + n;
                ab[0] = reduce_sum(a128[ib][c][0], q, qi);
                ab[LN] = reduce_sum(a128[ib][c][1], q, qi);
            }
        }
    }
    return ok;
}

// ---- column arithmetic ----------------------------------------------------------------------
// A residue x < 2^60 is split as x = x0 + x1 2^30 (x0, x1 < 2^30).  The product of two such
// residues is four 32 x 32 -> 64-bit partial products (one mad.wide.u32 each) summed into three
// 64-bit columns: V = c0 + c1 2^30 + c2 2^60 with c0 += x0 y0, c1 += x0 y1 + x1 y0, c2 += x1 y1.
// No carry chain: the columns have headroom (each partial product is below 2^60) and are
// normalised (fold) before they could overflow.
constexpr uint32_t kM30 = (1u << 30) - 1;

struct Cols {
    uint64_t c0, c1, c2;
};

__device__ __forceinline__ void madw(uint64_t& acc, uint32_t a, uint32_t b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

__device__ __forceinline__ void cmac(Cols& a, uint32_t x0, uint32_t x1, uint32_t y0, uint32_t y1) {
    madw(a.c0, x0, y0);
    madw(a.c1, x0, y1);
    madw(a.c1, x1, y0);
    madw(a.c2, x1, y1);
}

__device__ __forceinline__ uint32_t lo30(uint64_t x) { return (uint32_t)x & kM30; }
__device__ __forceinline__ uint32_t hi30(uint64_t x) { return (uint32_t)(x >> 30); }

// Carries c0 -> c1 -> c2 and reduces c2 modulo q (c2 counts multiples of 2^60, so c2 mod q
// changes V by a multiple of q): afterwards c0, c1 < 2^30 + 2^34 and c2 < 2^60 + 16 (2^60 - q).
__device__ __forceinline__ void fold(Cols& a, uint64_t q) {
    a.c1 += a.c0 >> 30;
    a.c0 &= kM30;
    a.c2 += a.c1 >> 30;
    a.c1 &= kM30;
    a.c2 -= (a.c2 >> 60) * q;
}

// Montgomery reduction by 2^60 in two 30-bit steps: returns r = (V + m q) / 2^60 = V 2^-60
// mod q, with r < V / 2^60 + q.  qi = -q^-1 mod 2^32 (only its low 30 bits matter).
// Requires c0 + 2^60 and c1 + 2^60 + 2^34 and c2 + 2^60 + 2^34 below 2^64.
__device__ __forceinline__ uint64_t mont60(Cols a, uint32_t q0, uint32_t q1, uint32_t qi) {
    uint32_t m = ((uint32_t)a.c0 * qi) & kM30;
    madw(a.c0, m, q0);                       // now a multiple of 2^30
    madw(a.c1, m, q1);
    a.c1 += a.c0 >> 30;
    m = ((uint32_t)a.c1 * qi) & kM30;
    madw(a.c1, m, q0);
    madw(a.c2, m, q1);
    return a.c2 + (a.c1 >> 30);
}

// x < 2^63 -> x mod q for q >= 2^55.  near60 (q > 2^63 / 9, as the special primes just below
// 2^60 are): x - floor(x / 2^60) q is below 2^60 + 7 (2^60 - q) < 2q, then one conditional
// subtraction; otherwise (x < 2^8 q) conditional subtractions of q 2^7 .. q.
__device__ __forceinline__ uint64_t below_q(uint64_t x, uint64_t q, bool near60) {
    if (near60) {
        x -= (x >> 60) * q;
        return x >= q ? x - q : x;
    }
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        const uint64_t m = q << i;
        x = x >= m ? x - m : x;
    }
    return x;
}

// 16 x mod q for x < q: a shift when 16 q < 2^60 (q < 2^56), else four modular doublings.
__device__ __forceinline__ uint64_t times16(uint64_t x, uint64_t q, bool small) {
    if (small) return x << 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) x = add_mod(x, x, q);
    return x;
}

// The tap sums' final reduction: V (normalised columns) -> V 2^-68 mod q in [0, q).
__device__ __forceinline__ uint64_t finish_cols(Cols a, uint64_t q, uint64_t qinv_neg,
                                                uint32_t q0, uint32_t q1, bool small, bool near60) {
    fold(a, q);
    uint64_t r = mont60(a, q0, q1, (uint32_t)qinv_neg);   // < 2^62
    if (small) {
        while (r >= q) r -= q;                 // r < 2^56 + q: a few subtractions at most
    } else {
        r = below_q(r, q, near60);
    }
    // times 2^-8: (r + m q) / 2^8 with m = -r q^-1 mod 2^8, below (q + 255 q) / 2^8 = q
    const uint64_t m = (r * qinv_neg) & 255u;
    U128 x{r, 0};
    mac128(x, m, q);
    return (x.lo >> 8) | (x.hi << 56);
}

// Compute warps, column arithmetic.  The keys are in Montgomery form (k 2^64), so a tap's key
// inner product reduced by mont60 is 16 (sum_j D_j k_j) mod q (the sum times 2^64 - 60); the
// P c0 term is brought to the same factor, and so is the key-less tap's P x.  The plaintexts
// are in Montgomery form too (p 2^64): the tap sums then carry 2^(4 + 64), and finish_cols
// divides by 2^68 (mont60 and one 8-bit step), giving exactly the chain version's residues.
// Operand bounds: keys, digits, P x and plaintexts are below q; x' (a tap's reduced value) is
// kept below 2^60 so that its halves are 30-bit.
template <int DNUM, int TILE>
__device__ __forceinline__ bool compute_cols(const uint64_t* __restrict__ smem, uint64_t* full, uint64_t* empty,
                                   const uint64_t* __restrict__ XPg, const TapTable& tt, int c_lo,
                                   int c_cnt, uint64_t* __restrict__ A, int b0, int nb, int l, int L,
                                   int n0, size_t LN, size_t LNq, int N, int logN, const ModConst& M,
                                   uint32_t report_polls) {
    using S = Stage<DNUM, TILE>;
    constexpr int kTile = S::T;
    const int tid = threadIdx.x;
    const bool qlimb = l < L;
    const uint64_t q = M.q;
    const uint32_t q0 = lo30(q), q1 = hi30(q), qi = (uint32_t)M.qinv_neg;
    const bool small = (q >> 55) == 0;        // q < 2^55: x' = r + 16 P c0 stays below 2^60
    const bool near60 = q > (1ull << 63) / 9;
    const int n = n0 + tid;
    bool ok = true;
    Cols acc[2][2][2];
#pragma unroll
    for (int ib = 0; ib < 2; ++ib)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int k = 0; k < 2; ++k) acc[ib][c][k] = Cols{0, 0, 0};
    for (int t = 0; t < tt.n; ++t) {
        const int s = t % kStages;
        const uint64_t* st = smem + s * S::WORDS;
        if (!mbar_wait(&full[s], (uint32_t)(t / kStages) & 1u, report_polls)) {
            ok = false;
            mbar_wait(&full[s], (uint32_t)(t / kStages) & 1u);
        }
        uint64_t x[2][2];                              // x' of each image and polynomial
        if (!tt.key[t]) {
#pragma unroll
            for (int ib = 0; ib < 2; ++ib)
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    x[ib][k] = (qlimb && ib < nb)
                                   ? times16(st[S::XP + (ib * 2 + k) * kTile + tid], q, small)
                                   : 0;
        } else {
            const uint32_t pn = perm_src((uint32_t)n, tt.g[t], logN);
            const int loc = (int)(pn & (kTile - 1));
            uint64_t xp[2] = {0, 0};                   // (P c0)[perm_g(n)] of each image
            if (qlimb) {
#pragma unroll
                for (int ib = 0; ib < 2; ++ib)
                    if (ib < nb)
                        xp[ib] = __ldg(XPg + ((size_t)(b0 + ib) * tt.n_sub + tt.sub[t]) * 2 * LNq +
                                       (size_t)l * N + pn);
            }
            uint32_t k0[DNUM][2], k1[DNUM][2];
#pragma unroll
            for (int j = 0; j < DNUM; ++j)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint64_t kv = st[S::KEYS + (2 * j + k) * kTile + tid];
                    k0[j][k] = lo30(kv);
                    k1[j][k] = hi30(kv);
                }
#pragma unroll
            for (int ib = 0; ib < 2; ++ib) {
                if (ib >= nb) {
                    x[ib][0] = x[ib][1] = 0;
                    continue;
                }
                Cols s0{0, 0, 0}, s1{0, 0, 0};
#pragma unroll
                for (int j = 0; j < DNUM; ++j) {
                    const uint64_t d = st[S::DIG + (ib * DNUM + j) * kTile + loc];
                    const uint32_t d0 = lo30(d), d1 = hi30(d);
                    cmac(s0, d0, d1, k0[j][0], k1[j][0]);
                    cmac(s1, d0, d1, k0[j][1], k1[j][1]);
                    if ((j & 3) == 3 && j + 1 < DNUM) {  // four digits: c1 < 2^63
                        fold(s0, q);
                        fold(s1, q);
                    }
                }
                uint64_t r0 = mont60(s0, q0, q1, qi), r1 = mont60(s1, q0, q1, qi);
                if (small) {                           // r < 2^56: no reduction needed
                    r0 += xp[ib] << 4;                 // + 16 (P c0), zero on special primes
                } else {
                    r0 = below_q(r0, q, near60);
                    r1 = below_q(r1, q, near60);
                    if (xp[ib]) r0 = add_mod(r0, times16(xp[ib], q, false), q);
                }
                x[ib][0] = r0;
                x[ib][1] = r1;
            }
        }
        const uint64_t pa = st[S::PTS + tid];
        const uint64_t pb = c_cnt > 1 ? st[S::PTS + kTile + tid] : 0;
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);   // this warp's last read of stage s
        const uint32_t pa0 = lo30(pa), pa1 = hi30(pa), pb0 = lo30(pb), pb1 = hi30(pb);
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const uint32_t x0 = lo30(x[ib][k]), x1 = hi30(x[ib][k]);
                cmac(acc[ib][0][k], x0, x1, pa0, pa1);
                if (c_cnt > 1) cmac(acc[ib][1][k], x0, x1, pb0, pb1);
            }
        if ((t & 3) == 3) {                            // every four taps: c1 < 2^63 + 2^34
#pragma unroll
            for (int ib = 0; ib < 2; ++ib)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int k = 0; k < 2; ++k) fold(acc[ib][c][k], q);
        }
    }
    if (ok) {
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) {
            if (ib >= nb) break;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c >= c_cnt) break;
                uint64_t* ab = A + (((size_t)(b0 + ib) * tt.r + c_lo + c) * 2) * LN + (size_t)l * N + n;
                ab[0] = finish_cols(acc[ib][c][0], q, M.qinv_neg, q0, q1, small, near60);
                ab[LN] = finish_cols(acc[ib][c][1], q, M.qinv_neg, q0, q1, small, near60);
            }
        }
    }
    return ok;
}

// ---- precomputed plaintext x key products (the ciphertext-prime limbs) ---------------------
// For a limb whose prime is below 2^50 the tap sum is rewritten with the products
// PK[c][t][j][k] = pt[c][t] key_t[j][k] (per coefficient, Montgomery form, computed once per
// launch from the resident keys and the layer's plaintexts):
//   acc_k[c] = sum_t ( sum_j D_j[perm_t(n)] PK[c][t][j][k] + [k = 0] (P c0)[perm_t(n)] pt[c][t] )
// (the key-less centre tap: (P c_k)[n] pt[c][0]).  Every term is a product of two residues
// below 2^50, split at bit 25 into halves below 2^25: four mad.wide.u32 add it into three
// 64-bit columns V = c0 + c1 2^25 + c2 2^50, each partial product below 2^50.  With at most
// (8 + 1) 64 = 576 terms per sum the columns stay below 2^61 and V below 576 q^2 < q 2^64, so
// the whole sum is reduced once, by one Montgomery reduction (REDC, 2^-64) at the end, which
// removes the single 2^64 factor every term carries.  No reduction per tap.
constexpr uint32_t kM25 = (1u << 25) - 1;
constexpr int kPkTile = 128;                          // coefficients per CTA
constexpr int kPkImages = 4;                          // images per CTA, two per thread

__device__ __forceinline__ uint64_t split25(uint64_t x) {   // x < 2^50 -> lo | hi << 32
    return (x & kM25) | ((x >> 25) << 32);
}

__global__ void k_pk_prep(const uint64_t* __restrict__ pts, TapTable tt, int c_lo, int dnum,
                          uint64_t* __restrict__ PK, int L, int K, int logN,
                          const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    int z = blockIdx.z;                               // ((c t + t) dnum + j) 2 + k
    const int k = z & 1;
    z >>= 1;
    const int j = z % dnum;
    z /= dnum;
    const int t = z % tt.n, c = z / tt.n;
    const uint64_t* key = tt.key[t];
    if (!key) return;
    const size_t LN = (size_t)(L + K) * N;
    const ModConst M = mods[l];
    U128 x{0, 0};
    mac128(x, pts[((size_t)(c_lo + c) * tt.n + t) * LN + (size_t)l * N + n],
           key[(size_t)(2 * j + k) * LN + (size_t)l * N + n]);
    PK[(size_t)blockIdx.z * L * N + (size_t)l * N + n] = split25(redc(x, M.q, M.qinv_neg));
}

template <int DNUM>
struct PkStage {
    static constexpr int T = kPkTile;
    static constexpr int PK = 0;                                   // [2 c][DNUM][2 k][T]
    static constexpr int PT = 2 * DNUM * 2 * T;                    // [2 c][T]
    static constexpr int DIG = PT + 2 * T;                         // [4 img][DNUM][T]
    static constexpr int XP = DIG;                                 // key-less: [4 img][2 k][T]
    static constexpr int WORDS = DIG + (kPkImages * DNUM > 8 ? kPkImages * DNUM : 8) * T;
    static constexpr int STAGES = DNUM <= 4 ? 3 : 2;
};

template <int DNUM>
__device__ __forceinline__ void issue_pk_tap(uint64_t* st, uint64_t* bar, int t, const TapTable& tt,
                                             const uint64_t* __restrict__ D,
                                             const uint64_t* __restrict__ XPg,
                                             const uint64_t* __restrict__ PK,
                                             const uint64_t* __restrict__ pts, int c_lo,
                                             int c_cnt, int b0, int nb, int l, int L, int n0,
                                             size_t LN, int N, int logN) {
    using S = PkStage<DNUM>;
    constexpr int T = S::T;
    const int lane = threadIdx.x & 31;
    const bool keyed = tt.key[t] != nullptr;
    const uint32_t row = T * 8;
    const int src0 = keyed ? (int)(perm_src((uint32_t)n0, tt.g[t], logN) & ~(uint32_t)(T - 1)) : n0;
    const int npk = keyed ? c_cnt * DNUM * 2 : 0;
    const int npt = c_cnt;
    const int ndig = keyed ? nb * DNUM : nb * 2;     // digit rows, or P x rows of the centre tap
    const int total = npk + npt + ndig;
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)total * row);
    __syncwarp();
    const size_t LNq = (size_t)L * N;
    for (int i = lane; i < total; i += 32) {
        uint64_t* dst;
        const uint64_t* src;
        if (i < npk) {                                // i = (c DNUM + j) 2 + k
            dst = st + S::PK + i * T;
            src = PK + ((size_t)(i / (2 * DNUM)) * tt.n * DNUM * 2 + (size_t)t * DNUM * 2 +
                        i % (2 * DNUM)) * LNq + (size_t)l * N + n0;
        } else if (i < npk + npt) {
            const int c = i - npk;
            dst = st + S::PT + c * T;
            src = pts + ((size_t)(c_lo + c) * tt.n + t) * LN + (size_t)l * N + n0;
        } else if (keyed) {
            const int q = i - npk - npt, ib = q / DNUM, j = q - ib * DNUM;
            const size_t it = (size_t)(b0 + ib) * tt.n_sub + tt.sub[t];
            dst = st + S::DIG + (ib * DNUM + j) * T;
            src = D + (it * DNUM + j) * LN + (size_t)l * N + src0;
        } else {
            const int q = i - npk - npt, ib = q >> 1, k = q & 1;
            const size_t it = (size_t)(b0 + ib) * tt.n_sub + tt.sub[t];
            dst = st + S::XP + (ib * 2 + k) * T;
            src = XPg + (it * 2 + k) * LNq + (size_t)l * N + n0;
        }
        bulk_copy(dst, src, row, bar);
    }
}

__device__ __forceinline__ void cmac25(Cols& a, uint32_t x0, uint32_t x1, uint32_t y0, uint32_t y1) {
    madw(a.c0, x0, y0);
    madw(a.c1, x0, y1);
    madw(a.c1, x1, y0);
    madw(a.c2, x1, y1);
}

// V = c0 + c1 2^25 + c2 2^50 (< q 2^64) -> V 2^-64 mod q.
__device__ __forceinline__ uint64_t finish25(const Cols& a, uint64_t q, uint64_t qinv_neg) {
    U128 v{a.c0, 0};
    uint64_t lo = a.c1 << 25, hi = a.c1 >> 39;
    v.lo += lo;
    v.hi += hi + (v.lo < lo);
    lo = a.c2 << 50;
    hi = a.c2 >> 14;
    v.lo += lo;
    v.hi += hi + (v.lo < lo);
    return redc(v, q, qinv_neg);
}

// One CTA: 128 coefficients of one ciphertext-prime limb for four images; compute thread
// tid < 256 holds coefficient n0 + (tid mod 128) of images 2 (tid / 128) and 2 (tid / 128) + 1.
// The last warp stages every tap's rows (PK, plaintexts, the digits of the permuted block or
// the centre tap's P x rows) with bulk copies, as in k_ks_mac_ext_bulk.
template <int DNUM>
__global__ void __launch_bounds__(2 * kPkTile + 32, DNUM <= 4 ? 2 : 1)
k_tap_pk(const uint64_t* __restrict__ D, const uint64_t* __restrict__ XPg,
         const uint64_t* __restrict__ PK, const uint64_t* __restrict__ pts, TapTable tt, int c_lo,
         int c_cnt, int B, uint64_t* __restrict__ A, int L, int K, int logN,
         const ModConst* __restrict__ mods, int* __restrict__ err, uint32_t report_polls) {
    using S = PkStage<DNUM>;
    constexpr int T = S::T;
    constexpr int kSt = S::STAGES;
    constexpr int kComputeWarps = 2 * T / 32;
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ __align__(8) uint64_t full[kSt], empty[kSt];
    const int N = 1 << logN;
    const int tid = threadIdx.x;
    const int n0 = blockIdx.y * T;
    const int l = blockIdx.z;
    const int b0 = blockIdx.x * kPkImages;
    const int nb = B - b0 < kPkImages ? B - b0 : kPkImages;
    const size_t LN = (size_t)(L + K) * N;
    const size_t LNq = (size_t)L * N;
    if (tid == 0) {
        for (int s = 0; s < kSt; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kComputeWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool ok = true;
    if (tid >= 2 * T) {                               // the producer warp
        for (int t = 0; t < tt.n; ++t) {
            const int s = t % kSt;
            if (t >= kSt) {
                ok &= mbar_wait(&empty[s], (uint32_t)((t / kSt) - 1) & 1u);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            issue_pk_tap<DNUM>(smem + s * S::WORDS, &full[s], t, tt, D, XPg, PK, pts, c_lo, c_cnt,
                               b0, nb, l, L, n0, LN, N, logN);
        }
    } else {
        const ModConst M = mods[l];
        const int col = tid & (T - 1);
        const int n = n0 + col;
        const int i0 = 2 * (tid / T);                 // this thread's first image in the CTA
        Cols acc[2][2][2];
#pragma unroll
        for (int ii = 0; ii < 2; ++ii)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int k = 0; k < 2; ++k) acc[ii][c][k] = Cols{0, 0, 0};
        // (P c0)[perm_t(n)] of this thread's images, loaded one keyed tap ahead of its use
        auto load_xp = [&](int t, uint64_t (&xp)[2]) {
            const uint32_t pn = perm_src((uint32_t)n, tt.g[t], logN);
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const int ib = i0 + ii;
                xp[ii] = (tt.key[t] && ib < nb)
                             ? __ldg(XPg + ((size_t)(b0 + ib) * tt.n_sub + tt.sub[t]) * 2 * LNq +
                                     (size_t)l * N + pn)
                             : 0;
            }
        };
        uint64_t xp_next[2];
        load_xp(0, xp_next);
        for (int t = 0; t < tt.n; ++t) {
            const int s = t % kSt;
            const uint64_t* st = smem + s * S::WORDS;
            const uint64_t xp_cur[2] = {xp_next[0], xp_next[1]};
            if (t + 1 < tt.n) load_xp(t + 1, xp_next);
            if (!mbar_wait(&full[s], (uint32_t)(t / kSt) & 1u, report_polls)) {
                ok = false;
                mbar_wait(&full[s], (uint32_t)(t / kSt) & 1u);
            }
            if (tt.key[t]) {
                const uint32_t pn = perm_src((uint32_t)n, tt.g[t], logN);
                const int loc = (int)(pn & (T - 1));
                uint32_t d0[2][DNUM], d1[2][DNUM], x0[2], x1[2];
#pragma unroll
                for (int ii = 0; ii < 2; ++ii) {
                    const int ib = i0 + ii;
                    const bool live = ib < nb;
                    const uint64_t xp = xp_cur[ii];
                    x0[ii] = (uint32_t)xp & kM25;
                    x1[ii] = (uint32_t)(xp >> 25);
#pragma unroll
                    for (int j = 0; j < DNUM; ++j) {
                        const uint64_t d = live ? st[S::DIG + (ib * DNUM + j) * T + loc] : 0;
                        d0[ii][j] = (uint32_t)d & kM25;
                        d1[ii][j] = (uint32_t)(d >> 25);
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c >= c_cnt) break;
                    const uint64_t p = st[S::PT + c * T + col];
                    const uint32_t p0 = (uint32_t)p & kM25, p1 = (uint32_t)(p >> 25);
#pragma unroll
                    for (int ii = 0; ii < 2; ++ii) cmac25(acc[ii][c][0], x0[ii], x1[ii], p0, p1);
#pragma unroll
                    for (int j = 0; j < DNUM; ++j)
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const uint64_t w = st[S::PK + ((c * DNUM + j) * 2 + k) * T + col];
                            const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
#pragma unroll
                            for (int ii = 0; ii < 2; ++ii)
                                cmac25(acc[ii][c][k], d0[ii][j], d1[ii][j], w0, w1);
                        }
                }
            } else {
                uint32_t x0[2][2], x1[2][2];
#pragma unroll
                for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int ib = i0 + ii;
                        const uint64_t x = ib < nb ? st[S::XP + (ib * 2 + k) * T + col] : 0;
                        x0[ii][k] = (uint32_t)x & kM25;
                        x1[ii][k] = (uint32_t)(x >> 25);
                    }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c >= c_cnt) break;
                    const uint64_t p = st[S::PT + c * T + col];
                    const uint32_t p0 = (uint32_t)p & kM25, p1 = (uint32_t)(p >> 25);
#pragma unroll
                    for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                        for (int k = 0; k < 2; ++k) cmac25(acc[ii][c][k], x0[ii][k], x1[ii][k], p0, p1);
                }
            }
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);   // this warp's last read of stage s
        }
        if (ok) {
#pragma unroll
            for (int ii = 0; ii < 2; ++ii) {
                const int ib = i0 + ii;
                if (ib >= nb) break;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c >= c_cnt) break;
                    uint64_t* ab = A + (((size_t)(b0 + ib) * tt.r + c_lo + c) * 2) * LN + (size_t)l * N + n;
                    ab[0] = finish25(acc[ii][c][0], M.q, M.qinv_neg);
                    ab[LN] = finish25(acc[ii][c][1], M.q, M.qinv_neg);
                }
            }
        }
    }
    if (!ok) atomicOr(err, 1);
    __syncthreads();
    if (!ok) {
        for (int s = 0; s < kSt && s < tt.n; ++s) {
            const int last = s + kSt * ((tt.n - 1 - s) / kSt);
            mbar_wait(&full[s], (uint32_t)(last / kSt) & 1u);
        }
    }
}

template <int DNUM, int TILE, int ARITH>
__global__ void __launch_bounds__(TILE + 32, min_ctas(DNUM, TILE, ARITH))
k_ks_mac_ext_bulk(const uint64_t* __restrict__ D, const uint64_t* __restrict__ XPg,
                  const uint64_t* __restrict__ pts, TapTable tt, int c_lo, int c_cnt, int B,
                  uint64_t* __restrict__ A, int L, int K, int logN,
                  const ModConst* __restrict__ mods, int* __restrict__ err,
                  uint32_t report_polls, int l0) {
    using S = Stage<DNUM, TILE>;
    constexpr int kTile = S::T;
    constexpr int kComputeWarps = kTile / 32;
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    const int N = 1 << logN;
    const int tid = threadIdx.x;
    const int n0 = blockIdx.y * kTile;
    const int l = l0 + blockIdx.z;                    // limbs l0 .. l0 + gridDim.z - 1
    const int b0 = blockIdx.x * 2;
    const int nb = B - b0 < 2 ? B - b0 : 2;
    const int LK = L + K;
    const size_t LN = (size_t)LK * N;
    const size_t LNq = (size_t)L * N;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);                 // the producer's expect_tx arrival + bytes
            mbar_init(&empty[s], kComputeWarps);    // one arrival per compute warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // a wait that runs out does not leave its loop (the other side would then wait too): the
    // thread goes on and the error bit makes the result unusable
    bool ok = true;
    if (tid >= kTile) {                               // the producer warp
        for (int t = 0; t < tt.n; ++t) {
            const int s = t % kStages;
            if (t >= kStages) {                       // every compute warp is done with tap t - 3
                ok &= mbar_wait(&empty[s], (uint32_t)((t / kStages) - 1) & 1u);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            issue_tap<DNUM, TILE>(smem + s * S::WORDS, &full[s], t, tt, D, XPg, pts, c_lo, c_cnt,
                                  b0, nb, l, L, n0, LN, N, logN);
        }
    } else if (ARITH == 0) {
        ok = compute_chain<DNUM, TILE>(smem, full, empty, XPg, tt, c_lo, c_cnt, A, b0, nb, l, L, n0,
                                       LN, LNq, N, logN, mods[l], report_polls);
    } else {
        ok = compute_cols<DNUM, TILE>(smem, full, empty, XPg, tt, c_lo, c_cnt, A, b0, nb, l, L, n0,
                                      LN, LNq, N, logN, mods[l], report_polls);
    }
    if (!ok) atomicOr(err, 1);
    __syncthreads();
    if (!ok) {
        // let this CTA's copies land before its shared memory is released (bounded): the last
        // tap staged in each stage
        for (int s = 0; s < kStages && s < tt.n; ++s) {
            const int last = s + kStages * ((tt.n - 1 - s) / kStages);
            mbar_wait(&full[s], (uint32_t)(last / kStages) & 1u);
        }
    }
}

template <int DNUM, int TILE, int ARITH>
void launch_bulk(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                 const TapTable& tt, uint64_t* A, int B, int c_lo, int cnt, int l0 = 0,
                 int n_limbs = -1) {
    const size_t smem = (size_t)kStages * Stage<DNUM, TILE>::WORDS * 8;
    static bool attr_set[64] = {};   // per template instance and device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(k_ks_mac_ext_bulk<DNUM, TILE, ARITH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const dim3 grid((B + 1) / 2, c->N / TILE, n_limbs < 0 ? c->L + c->K : n_limbs);
    k_ks_mac_ext_bulk<DNUM, TILE, ARITH><<<grid, TILE + 32, smem, c->stream>>>(
        D, XP, pts, tt, c_lo, cnt, B, A, c->L, c->K, c->logN, c->d_mod, c->d_err,
        c->wait_report >= 0 ? (uint32_t)c->wait_report : kWaitSpins, l0);
}

// Precomputed products: PK for the channel pair, the ciphertext-prime limbs by k_tap_pk, the
// special-prime limbs by the carry-chain kernel.
template <int DNUM>
void launch_pk(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
               const TapTable& tt, uint64_t* A, int B, int c_lo, int cnt, uint64_t* PK) {
    ++c->launches;
    const dim3 gp((c->N + 255) / 256, c->L, cnt * tt.n * DNUM * 2);
    k_pk_prep<<<gp, 256, 0, c->stream>>>(pts, tt, c_lo, DNUM, PK, c->L, c->K, c->logN, c->d_mod);
    using S = PkStage<DNUM>;
    const size_t smem = (size_t)S::STAGES * S::WORDS * 8;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(k_tap_pk<DNUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    ++c->launches;
    const dim3 grid((B + kPkImages - 1) / kPkImages, c->N / kPkTile, c->L);
    k_tap_pk<DNUM><<<grid, 2 * kPkTile + 32, smem, c->stream>>>(
        D, XP, PK, pts, tt, c_lo, cnt, B, A, c->L, c->K, c->logN, c->d_mod, c->d_err,
        c->wait_report >= 0 ? (uint32_t)c->wait_report : kWaitSpins);
    ++c->launches;
    launch_bulk<DNUM, 128, 0>(c, D, XP, pts, tt, A, B, c_lo, cnt, c->L, c->K);
}

template <int DNUM>
void launch_pk_pairs(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                     const TapTable& tt, uint64_t* A, int B, uint64_t* PK) {
    for (int c_lo = 0; c_lo < tt.r; c_lo += 2) {
        const int cnt = tt.r - c_lo < 2 ? tt.r - c_lo : 2;
        launch_pk<DNUM>(c, D, XP, pts, tt, A, B, c_lo, cnt, PK);
    }
}

template <int TILE, int ARITH>
void launch_bulk_tile(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                      const TapTable& tt, uint64_t* A, int B, int c_lo, int cnt) {
    switch (c->dnum) {
        case 1: launch_bulk<1, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 2: launch_bulk<2, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 3: launch_bulk<3, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 4: launch_bulk<4, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 5: launch_bulk<5, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 6: launch_bulk<6, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        case 7: launch_bulk<7, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
        default: launch_bulk<8, TILE, ARITH>(c, D, XP, pts, tt, A, B, c_lo, cnt); break;
    }
}

}  // namespace

bool tapmac_bulk_supported(const he_ctx* c) { return c->N >= kMaxTile && c->dnum <= 8; }

// The precomputed-product path needs every ciphertext prime below 2^50 (25-bit halves).
static bool pk_supported(const he_ctx* c) {
    if (!tapmac_bulk_supported(c)) return false;
    for (int i = 0; i < c->L; ++i)
        if (c->mods[i] >> 50) return false;
    return true;
}

// Its product buffer for one channel pair: [2][taps][dnum][2][L][N] words.  Grown outside a
// recording only; NULL (the chain path is used instead) if it cannot be had.
static uint64_t* pk_buffer(he_ctx* c, const TapTable& tt) {
    const size_t words = (size_t)2 * tt.n * c->dnum * 2 * c->L * c->N;
    if (words * 8 + 4096 > c->pk.cap && (c->rec || pk_reserve(c, words))) return nullptr;
    return (uint64_t*)c->pk.base;
}

void launch_ks_mac_ext_bulk(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                            const TapTable& tt, uint64_t* A, int B) {
    if (c->tap_arith == 2 && pk_supported(c)) {
        if (uint64_t* PK = pk_buffer(c, tt)) {
            switch (c->dnum) {
                case 1: launch_pk_pairs<1>(c, D, XP, pts, tt, A, B, PK); return;
                case 2: launch_pk_pairs<2>(c, D, XP, pts, tt, A, B, PK); return;
                case 3: launch_pk_pairs<3>(c, D, XP, pts, tt, A, B, PK); return;
                case 4: launch_pk_pairs<4>(c, D, XP, pts, tt, A, B, PK); return;
                case 5: launch_pk_pairs<5>(c, D, XP, pts, tt, A, B, PK); return;
                case 6: launch_pk_pairs<6>(c, D, XP, pts, tt, A, B, PK); return;
                case 7: launch_pk_pairs<7>(c, D, XP, pts, tt, A, B, PK); return;
                default: launch_pk_pairs<8>(c, D, XP, pts, tt, A, B, PK); return;
            }
        }
    }
    const int tile = c->tap_tile ? c->tap_tile : default_tile(c->dnum);
    for (int c_lo = 0; c_lo < tt.r; c_lo += 2) {
        ++c->launches;
        const int cnt = tt.r - c_lo < 2 ? tt.r - c_lo : 2;
        const bool cols = c->tap_arith != 0;
        if (tile == 128) {
            if (cols) launch_bulk_tile<128, 1>(c, D, XP, pts, tt, A, B, c_lo, cnt);
            else launch_bulk_tile<128, 0>(c, D, XP, pts, tt, A, B, c_lo, cnt);
        } else {
            if (cols) launch_bulk_tile<256, 1>(c, D, XP, pts, tt, A, B, c_lo, cnt);
            else launch_bulk_tile<256, 0>(c, D, XP, pts, tt, A, B, c_lo, cnt);
        }
    }
}

// Autotuner: times the NTT splits worth trying on a batch's ciphertexts (forward and inverse)
// and both tap-kernel tiles on synthetic operands of `batch` images (25 taps, 2 channels, the
// context's key shape), and keeps the fastest of each for this context.
static int tune_ntt(he_ctx* ctx, int batch, double* best_ms) {
    int cand[4];
    const int nc = ntt_split_candidates(ctx->logN, cand, 4);
    const size_t items = (size_t)2 * batch, n = items * ctx->L * ctx->N;
    int rc = arena_reserve(ctx, n + 32);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, n);
    for (size_t it = 0; it < items; ++it)
        launch_uniform(ctx, he_stream_state(0x6e7474ull, it), X + it * ctx->L * ctx->N, ctx->L, 0, 0);
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    double best = 1e30;
    int best_s1 = cand[0], best_radix = 3;
    for (int v = 0; v < 2 * nc; ++v) {                 // every split at radix 8, then radix 4
        const int c = v % nc;
        ctx->ntt_s1 = cand[c];
        ctx->ntt_radix = v < nc ? 3 : 2;
        ntt_prepare(ctx);
        ntt_forward(ctx, X, (int)items, (size_t)ctx->L * ctx->N, ctx->L, 0);     // warm-up
        ntt_inverse(ctx, X, (int)items, (size_t)ctx->L * ctx->N, ctx->L, 0);
        cudaEventRecord(e0, ctx->stream);
        for (int rep = 0; rep < 3; ++rep) {
            ntt_forward(ctx, X, (int)items, (size_t)ctx->L * ctx->N, ctx->L, 0);
            ntt_inverse(ctx, X, (int)items, (size_t)ctx->L * ctx->N, ctx->L, 0);
        }
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t / 3.0 < best) {
            best = t / 3.0;
            best_s1 = cand[c];
            best_radix = ctx->ntt_radix;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->ntt_s1 = best_s1;
    ctx->ntt_radix = best_radix;
    ntt_prepare(ctx);
    *best_ms = best;
    return he_launch_check(ctx, "he_autotune");
}

// Limb groups of the ModUp / ModDown base conversions: both conversions timed on synthetic
// operands of `batch` ciphertexts with the target limbs split over 1, 2 and 4 groups.
static int tune_limb_groups(he_ctx* ctx, int batch, double* ms) {
    const size_t N = ctx->N, L = ctx->L, LK = ctx->L + ctx->K, dn = ctx->dnum;
    const size_t nX = (size_t)batch * 2 * L * N, nD = (size_t)batch * dn * LK * N,
                 nU = (size_t)batch * 2 * LK * N, nV = (size_t)batch * 2 * L * N;
    int rc = arena_reserve(ctx, nX + nD + nU + nV + 32 * 4);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, nX);
    uint64_t* D = arena_take(ctx, nD);
    uint64_t* U = arena_take(ctx, nU);
    uint64_t* V = arena_take(ctx, nV);
    for (int b = 0; b < batch; ++b) {
        launch_uniform(ctx, he_stream_state(0x6c696d62ull, 2 * b), X + (size_t)b * 2 * L * N, (int)L, 0, 0);
        launch_uniform(ctx, he_stream_state(0x6c696d62ull, 2 * b + 1), U + (size_t)b * 2 * LK * N, (int)LK, 0, 0);
    }
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    const int cand[3] = {1, 2, 4};
    int best = 0;
    for (int v = 0; v < 3; ++v) {
        ctx->limb_groups = cand[v];
        auto run = [&]() {
            launch_modup(ctx, X, 2 * L * N, X + L * N, 2 * L * N, 1u, D, dn * LK * N, batch);
            launch_moddown_conv(ctx, U, 2 * LK * N, V, 2 * L * N, batch);
        };
        run();
        cudaEventRecord(e0, ctx->stream);
        for (int rep = 0; rep < 3; ++rep) run();
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[v] = t / 3.0;
        if (ms[v] < ms[best]) best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->limb_groups = cand[best];
    return he_launch_check(ctx, "he_autotune");
}

// Where the ModUp / ModDown base conversions run: separate kernels (with the chosen limb
// groups) or inside the forward NTT's first pass.  Both timed as one ModUp and one ModDown of
// min(batch, 64) synthetic ciphertexts; ms[0] separate, ms[1] fused.
static int tune_bconv(he_ctx* ctx, int batch, double* ms) {
    const int items = std::min(batch, 64);
    const size_t N = ctx->N, L = ctx->L, ct = 2 * L * N;
    int rc = arena_reserve(ctx, items * ct + items * rot_scratch_per_item(ctx) + 64);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, items * ct);
    RotBufs b = rot_bufs_take(ctx, items);
    for (int it = 0; it < items; ++it) {
        launch_uniform(ctx, he_stream_state(0x62636f6eull, 2 * it), X + it * ct, (int)L, 0, 0);
        launch_uniform(ctx, he_stream_state(0x62636f6eull, 2 * it + 1), b.u + it * 2 * (L + ctx->K) * N,
                       (int)(L + ctx->K), 0, 0);
    }
    std::vector<uint64_t*> outs(items);
    for (int it = 0; it < items; ++it) outs[it] = X + it * ct;   // overwritten: fine for timing
    auto outp = upload_out_ptrs(ctx, outs);
    if (!outp) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    for (int v = 0; v < 2; ++v) {
        ctx->bconv_fused = v;
        auto run = [&]() {
            modup_items(ctx, X, items, 1u, b);
            moddown_combine(ctx, b.u, b.v, items, nullptr, nullptr, outp, 1u);
        };
        run();
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < 3; ++r) run();
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[v] = t / 3.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->bconv_fused = ms[1] <= ms[0] ? 1 : 0;
    return he_launch_check(ctx, "he_autotune");
}

extern "C" int he_autotune(he_ctx* ctx, int batch, int force_tile, double* ms_out) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_autotune");
    if (force_tile) {
        if (force_tile != 128 && force_tile != 256)
            return he_fail(ctx, HE_EINVAL, "he_autotune: tile must be 128 or 256");
        ctx->tap_tile = force_tile;
        return HE_OK;
    }
    if (batch < 1 || batch > 1024) return he_fail(ctx, HE_EINVAL, "he_autotune: batch out of range");
    double ntt_ms = 0, lg_ms[3] = {0, 0, 0};
    int rc = tune_ntt(ctx, batch, &ntt_ms);
    if (rc) return rc;
    if ((rc = tune_limb_groups(ctx, batch, lg_ms))) return rc;
    double bc_ms[2] = {0, 0};
    if ((rc = tune_bconv(ctx, batch, bc_ms))) return rc;
    if (ms_out) {
        for (int i = 0; i < HE_TUNE_REPORT_LEN; ++i) ms_out[i] = 0.0;
        ms_out[4] = ntt_ms;
        ms_out[5] = ctx->ntt_s1;
        ms_out[9] = 1 << ctx->ntt_radix;
        for (int v = 0; v < 3; ++v) ms_out[10 + v] = lg_ms[v];
        ms_out[13] = ctx->limb_groups;
        ms_out[14] = bc_ms[0];
        ms_out[15] = bc_ms[1];
        ms_out[6] = default_tile(ctx->dnum);
        ms_out[7] = ctx->tap_arith;
    }
    if (!tapmac_bulk_supported(ctx)) return HE_OK;        // no tile to choose
    const int L = ctx->L, LK = L + ctx->K, dn = ctx->dnum, taps = 25, r = 2;
    const size_t N = ctx->N, LN = (size_t)LK * N;
    const size_t nD = (size_t)batch * dn * LN, nXP = (size_t)batch * 2 * L * N,
                 nP = (size_t)r * taps * LN, nK = (size_t)dn * 2 * LN,
                 nA = (size_t)batch * r * 2 * LN;
    if ((rc = arena_reserve(ctx, nD + nXP + nP + nK + nA + 32 * 8))) return rc;
    arena_reset(ctx);
    uint64_t* D = arena_take(ctx, nD);
    uint64_t* XP = arena_take(ctx, nXP);
    uint64_t* P = arena_take(ctx, nP);
    uint64_t* Kb = arena_take(ctx, nK);
    uint64_t* A = arena_take(ctx, nA);
    // uniform residues, one counter stream per row block
    uint64_t blk = 0;
    auto fill = [&](uint64_t* p, size_t rows_total, int rows_per_block) {
        for (size_t r0 = 0; r0 < rows_total; r0 += rows_per_block)
            launch_uniform(ctx, he_stream_state(0x61757475ull, blk++), p + r0 * N, rows_per_block, 0, 0);
    };
    fill(D, (size_t)batch * dn * LK, LK);
    fill(XP, (size_t)batch * 2 * L, L);
    fill(P, (size_t)r * taps * LK, LK);
    fill(Kb, (size_t)dn * 2 * LK, LK);
    TapTable tt{};
    tt.n = taps;
    tt.r = r;
    tt.n_sub = 1;
    for (int t = 0; t < taps; ++t) {
        tt.key[t] = t ? Kb : nullptr;
        tt.g[t] = t ? galois_elt(ctx, t) : 1u;
    }
    // every (tile, arithmetic) pair, timed on the same operands, then the precomputed-product
    // path (its own tiling: 128 coefficients, four images per CTA)
    const int tiles[2] = {128, 256};
    double ms[5] = {0, 0, 0, 0, 0};
    cudaEvent_t e0, e1;
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e0));
    HE_CHECK_CUDA(ctx, cudaEventCreate(&e1));
    int best = 0;
    const int nv = pk_supported(ctx) ? 5 : 4;
    for (int v = 0; v < nv; ++v) {
        ctx->tap_tile = v == 4 ? 128 : tiles[v >> 1];
        ctx->tap_arith = v == 4 ? 2 : (v & 1);
        launch_ks_mac_ext_bulk(ctx, D, XP, P, tt, A, batch);          // warm-up
        cudaEventRecord(e0, ctx->stream);
        for (int rep = 0; rep < 3; ++rep) launch_ks_mac_ext_bulk(ctx, D, XP, P, tt, A, batch);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[v] = t / 3.0;
        if (ms[v] < ms[best]) best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tap_tile = best == 4 ? 128 : tiles[best >> 1];
    ctx->tap_arith = best == 4 ? 2 : (best & 1);
    if (ms_out) {
        for (int v = 0; v < 4; ++v) ms_out[v] = ms[v];
        ms_out[8] = ms[4];
        ms_out[6] = ctx->tap_tile;
        ms_out[7] = ctx->tap_arith;
    }
    return he_launch_check(ctx, "he_autotune");
}

extern "C" int he_set_wait_report(he_ctx* ctx, int polls) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_set_wait_report");
    ctx->wait_report = polls < 0 ? -1 : polls;
    return HE_OK;
}

extern "C" int he_tune_set(he_ctx* ctx, int knob, int value) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_tune_set");
    switch (knob) {
        case HE_TUNE_TAP_TILE:
            if (value != -1 && value != 128 && value != 256)
                return he_fail(ctx, HE_EINVAL, "he_tune_set: the tap tile is 128 or 256");
            ctx->tap_tile = value < 0 ? 0 : value;
            return HE_OK;
        case HE_TUNE_TAP_ARITH:
            if (value < -1 || value > 2)
                return he_fail(ctx, HE_EINVAL, "he_tune_set: tap arithmetic is 0 (chains), 1 "
                                               "(columns) or 2 (precomputed products)");
            ctx->tap_arith = value < 0 ? 0 : value;
            return HE_OK;
        case HE_TUNE_NTT_SPLIT:
            if (value != -1 && (value < 1 || value >= ctx->logN))
                return he_fail(ctx, HE_EINVAL, "he_tune_set: NTT split log2 N1 out of range");
            ctx->ntt_s1 = value < 0 ? 0 : value;
            ntt_prepare(ctx);
            return HE_OK;
        case HE_TUNE_NTT_RADIX:
            if (value != -1 && value != 4 && value != 8)
                return he_fail(ctx, HE_EINVAL, "he_tune_set: NTT radix is 4 or 8");
            ctx->ntt_radix = value < 0 ? 0 : (value == 8 ? 3 : 2);
            ntt_prepare(ctx);
            return HE_OK;
        case HE_TUNE_LIMB_GROUPS:
            if (value != -1 && value != 1 && value != 2 && value != 4)
                return he_fail(ctx, HE_EINVAL, "he_tune_set: limb groups are 1, 2 or 4");
            ctx->limb_groups = value < 0 ? 0 : value;
            return HE_OK;
        case HE_TUNE_BCONV_FUSED:
            if (value < -1 || value > 1)
                return he_fail(ctx, HE_EINVAL, "he_tune_set: base conversion placement is 0 "
                                               "(separate kernels) or 1 (inside the NTT)");
            ctx->bconv_fused = value < 0 ? 1 : value;
            return HE_OK;
        default:
            return he_fail(ctx, HE_EINVAL, "he_tune_set: unknown knob");
    }
}

extern "C" int he_tune_get(he_ctx* ctx, int knob, int* value) {
    if (!ctx || !value) return HE_EINVAL;
    switch (knob) {
        case HE_TUNE_TAP_TILE: *value = ctx->tap_tile ? ctx->tap_tile : default_tile(ctx->dnum); return HE_OK;
        case HE_TUNE_TAP_ARITH: *value = ctx->tap_arith; return HE_OK;
        case HE_TUNE_NTT_SPLIT: *value = ctx->ntt_s1 ? ctx->ntt_s1 : ctx->logN / 2; return HE_OK;
        case HE_TUNE_NTT_RADIX: *value = 1 << (ctx->ntt_radix ? ctx->ntt_radix : 3); return HE_OK;
        case HE_TUNE_LIMB_GROUPS: *value = ctx->limb_groups ? ctx->limb_groups : 1; return HE_OK;
        case HE_TUNE_BCONV_FUSED: *value = ctx->bconv_fused; return HE_OK;
        default: return he_fail(ctx, HE_EINVAL, "he_tune_get: unknown knob");
    }
}
