// ntt.cu -- negacyclic NTT / inverse NTT over Z_q[X]/(X^N+1), batched over limbs and items.
//
// Forward transform: merged-psi Cooley-Tukey, stage s (m = 2^s, t = N / 2^(s+1)) pairs
// (j, j+t) in group i = j / 2t with twiddle psi^brv(m + i); the output is in bit-reversed
// order, position p holding a(psi^(2 brv(p) + 1)).  Inverse: Gentleman-Sande with
// psi^-brv(m + i), stages in reverse, then the factor N^-1.
//
// The N = N1 N2 points (N1 = 2^s1, s1 chosen for the fewest rounds) are split in two passes:
//   column pass: stages s < s1 act on elements with the same j mod N2 (strided columns);
//                one CTA holds `cols` adjacent columns x N1 rows;
//   row pass:    stages s >= s1 act inside contiguous blocks of N2 elements; one CTA holds
//                `blocks` blocks.
// Inside a pass every thread keeps 8 residues in registers and applies up to three stages
// per round (a radix-8 step on one group of 8, or two radix-4 / four radix-2 groups): the
// elements of a group share all index bits except the round's K stage bits.  Rounds exchange
// through shared memory; the first round reads global memory directly and the last writes it.
// Butterflies use Harvey's lazy reduction: forward values stay in [0, 4q), inverse values in
// [0, 2q), and are brought to [0, q) at the end (moduli below 2^62).  Forward transforms of a
// modulus below 2^57 ("small") skip the per-butterfly reduction altogether and estimate the
// Shoup quotient from three partial products: each stage adds less than 4q to a value, so
// after at most 16 stages every value stays below 4q + 64q < 2^64, and the pass's last write
// reduces it exactly (a 32-bit quotient estimate and one conditional subtraction,
// reduce_small).  The output is the same residue in [0, q).
// Rounds hold up to 2^K elements per group with K <= the context's radix cap (log2 of 2, 4 or
// 8; the autotuner picks it).
#include "he_internal.cuh"

namespace {

constexpr int kTile = 2048;   // residues staged per CTA (16 KiB), 8 per thread

__device__ __forceinline__ void bfly_ct(uint64_t& X, uint64_t& Y, const ShoupPair& W, uint64_t q,
                                        uint64_t q2) {
    uint64_t x = X >= q2 ? X - q2 : X;               // [0, 2q)
    uint64_t t = mul_shoup_lazy(Y, W.w, W.ws, q);    // [0, 2q)
    X = x + t;                                       // [0, 4q)
    Y = x - t + q2;                                  // (0, 4q)
}

// Forward butterfly without reduction (small moduli): t in [0, 4q), X + t and X - t + 4q grow
// by less than 4q per stage.
__device__ __forceinline__ void bfly_ct_small(uint64_t& X, uint64_t& Y, const ShoupPair& W,
                                              uint64_t q, uint64_t q4) {
    const uint64_t t = mul_shoup_approx(Y, W.w, W.ws, q);
    const uint64_t x = X;
    X = x + t;
    Y = x - t + q4;
}

__device__ __forceinline__ void bfly_gs(uint64_t& X, uint64_t& Y, const ShoupPair& W, uint64_t q,
                                        uint64_t q2) {
    uint64_t s = X + Y;                              // X, Y in [0, 2q)
    s = s >= q2 ? s - q2 : s;
    uint64_t d = X - Y + q2;                         // (0, 4q)
    X = s;
    Y = mul_shoup_lazy(d, W.w, W.ws, q);             // [0, 2q)
}

// Inverse butterfly for q < 2^61: values kept in [0, 4q) (8q < 2^64), the Shoup product
// estimated from three partial products ([0, 4q) for any 64-bit input).  The pass's last
// product by N^-1 is a full Shoup product and brings every value to [0, q).
__device__ __forceinline__ void bfly_gs_small(uint64_t& X, uint64_t& Y, const ShoupPair& W,
                                              uint64_t q, uint64_t q4) {
    uint64_t s = X + Y;                              // < 8q
    s = s >= q4 ? s - q4 : s;                        // [0, 4q)
    const uint64_t d = X - Y + q4;                   // (0, 8q)
    X = s;
    Y = mul_shoup_approx(d, W.w, W.ws, q);           // [0, 4q)
}

// Butterflies of one round on the thread's 8 registers: (8 >> K) groups of 2^K elements,
// group g at x[g * 2^K + m].  Twiddle of stage ee for element m of a group whose block index
// is `hi` (plus the block offset `toff` of the row pass): psi^brv(2^s + toff 2^ee + hi 2^ee
// + (m >> (K - ee))).
// ROWT (the forward row pass): the reordered table, where stage s's entry (base, j) sits at
// 2^s + j 2^s0 + base (s0 the round's first stage): lanes with consecutive groups read
// consecutive entries.  (The inverse row pass measured slower with its own reordered table.)
template <int K, bool INV, bool SMALL, bool ROWT = false>
__device__ __forceinline__ void round_bflies(uint64_t (&x)[8], const int (&hi)[8 >> K], int s0,
                                             int toff, const ShoupPair* __restrict__ w,
                                             uint64_t q, uint64_t q2) {
    constexpr int M = 1 << K;
#pragma unroll
    for (int g = 0; g < (8 >> K); ++g) {
        const int base_hi = toff + hi[g];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int ee = INV ? (K - 1 - k) : k;
            const int d = 1 << (K - 1 - ee);
            const int s = s0 + ee;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (m & d) continue;
                // one 16-byte load per pair (the tables are 16-byte aligned): half the L1
                // wavefronts of two 8-byte loads
                const int ti = ROWT ? (1 << s) + ((m >> (K - ee)) << s0) + base_hi
                                    : (1 << s) + (base_hi << ee) + (m >> (K - ee));
                const ulonglong2 tw = __ldg(reinterpret_cast<const ulonglong2*>(w) + ti);
                const ShoupPair W{tw.x, tw.y};
                if (INV && SMALL) bfly_gs_small(x[g * M + m], x[g * M + m + d], W, q, 2 * q2);
                else if (INV) bfly_gs(x[g * M + m], x[g * M + m + d], W, q, q2);
                else if (SMALL) bfly_ct_small(x[g * M + m], x[g * M + m + d], W, q, 2 * q2);
                else bfly_ct(x[g * M + m], x[g * M + m + d], W, q, q2);
            }
        }
    }
}

// The fused base conversion as one CTA of the column pass sees it: the item's source limbs
// and the constants of the CTA's target modulus (staged in shared memory).
struct BConvCta {
    const uint64_t* s;
    const ShoupPair* c;
    int ns, N;
};

// One round of the column pass.  Element m of group Gi: column c = Gi mod cols, row
// hi (tlow 2^K) + m tlow + lo with (hi, lo) = divmod(Gi / cols, tlow).  cols = 2^lc and
// tlow = 2^(s1 - e0 - K), so the divisions are shifts.
template <int K, bool INV, bool SMALL, bool PRO>
__device__ __forceinline__ void col_round(uint64_t (&x)[8], uint64_t* sm, uint64_t* __restrict__ a,
                                          bool first, bool last, int e0, int s1, int N2, int lo0,
                                          int lc, const ShoupPair* __restrict__ w,
                                          const ModConst& Mc, const BConvCta& pc,
                                          const ShoupPair& osc) {
    constexpr int M = 1 << K;
    const int ltl = s1 - e0 - K, tlow = 1 << ltl;
    const int cmask = (1 << lc) - 1;
    const int nthr = blockDim.x, tid = threadIdx.x;
    int hi[8 >> K];
    int off[8];
#pragma unroll
    for (int g = 0; g < (8 >> K); ++g) {
        const int Gi = tid + g * nthr;
        const int c = Gi & cmask, Gc = Gi >> lc;
        hi[g] = Gc >> ltl;
        const int lo = Gc & (tlow - 1);
#pragma unroll
        for (int m = 0; m < M; ++m)
            off[g * M + m] = ((((hi[g] << K) + m) << ltl) + lo) << lc | c;
    }
    if (first && PRO) {
        // source limb by source limb, the thread's eight loads in flight together
        const uint64_t q = Mc.q;
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= pc.ns) break;
            const uint64_t* sk = pc.s + (size_t)k * pc.N + lo0;
            const ShoupPair ck = pc.c[k];
            uint64_t v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = sk[(size_t)(off[i] >> lc) * N2 + (off[i] & cmask)];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = add_mod(x[i], mul_shoup(v[i], ck.w, ck.ws, q), q);
        }
    } else if (first) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = off[i] >> lc, c = off[i] & cmask;
            x[i] = a[(size_t)row * N2 + lo0 + c];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = sm[off[i]];
    }
    const uint64_t q = Mc.q, q2 = 2 * q;
    round_bflies<K, INV, SMALL>(x, hi, e0, 0, w, q, q2);
    if (last) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = off[i] >> lc, c = off[i] & cmask;
            uint64_t v = x[i];
            if (INV) v = mul_shoup(v, osc.w, osc.ws, q);
            a[(size_t)row * N2 + lo0 + c] = v;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) sm[off[i]] = x[i];
        __syncthreads();
    }
}

// Shared-memory index of the row pass: word w goes to w ^ ((w >> 4) & 15), a permutation inside
// each row of 16 words (128 bytes, the 32 banks).  The later rounds' strided patterns (groups of
// 4 consecutive words 32 words apart, or words 4 apart) otherwise fall on 4 of the 16 bank
// pairs, 8-way conflicts; swizzled, every pattern of the pass spreads a warp's 32 words over all
// 16 pairs, two each (the minimum two wavefronts of a 64-bit access).
__device__ __forceinline__ int swz(int w) { return w ^ ((w >> 4) & 15); }

// The combine step as one CTA of the row pass sees it (CombineDst for its item and row).
struct CombineCta {
    const uint64_t* u;
    uint64_t* o;
    const uint64_t* c0;
    const uint64_t* base;
    ShoupPair pinv;
    uint32_t g;
};

// One round of the row pass.  Element m of group Gi: block b = Gi / (N2 >> K) of the tile,
// local index hi (tlow 2^K) + m tlow + lo.
template <int K, bool INV, bool SMALL, bool EPI>
__device__ __forceinline__ void row_round(uint64_t (&x)[8], uint64_t* sm, uint64_t* __restrict__ a,
                                          bool first, bool last, int e0, int s1, int s2, int blk0,
                                          const ShoupPair* __restrict__ w, const ModConst& Mc,
                                          const CombineCta& ep) {
    constexpr int M = 1 << K;
    const int N2 = 1 << s2;
    const int ltl = s2 - e0 - K, tlow = 1 << ltl;
    const int lpb = s2 - K;                       // log2 of the groups per block
    const int nthr = blockDim.x, tid = threadIdx.x;
    // all groups of one thread lie in the same block when per_blk >= nthr, else they differ:
    // keep the block of each group separately.
    int hi[8 >> K];
    int blk[8 >> K];
    int off[8];
#pragma unroll
    for (int g = 0; g < (8 >> K); ++g) {
        const int Gi = tid + g * nthr;
        const int b = Gi >> lpb, Gl = Gi & ((1 << lpb) - 1);
        hi[g] = Gl >> ltl;
        blk[g] = b;
        const int lo = Gl & (tlow - 1);
#pragma unroll
        for (int m = 0; m < M; ++m)
            off[g * M + m] = (b << s2) + ((((hi[g] << K) + m) << ltl) | lo);
    }
    // The forward pass ends with its shortest strides (a thread's 2^K residues adjacent): its
    // last round leaves through shared memory, so that global memory is written in whole lines
    // (the same staging at the inverse pass's start measured slower).
    const int tile = nthr * 8;
    uint64_t* at = a + (size_t)blk0 * N2;
    if (first) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = at[off[i]];
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = sm[swz(off[i])];
    }
    const uint64_t q = Mc.q, q2 = 2 * q;
    // twiddle offset of block (blk0 + b) at stage s1 + e0 + ee is (blk0 + b) 2^(e0 + ee):
    // fold it into hi as (blk0 + b) 2^e0 + hi.
    int hh[8 >> K];
#pragma unroll
    for (int g = 0; g < (8 >> K); ++g) hh[g] = ((blk0 + blk[g]) << e0) + hi[g];
    round_bflies<K, INV, SMALL, !INV>(x, hh, s1 + e0, 0, w, q, q2);
    if (last && !INV) {
        // reduced values back to the locations this thread read (no other thread reads them
        // in this round), then the tile leaves in order
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            uint64_t v = x[i];
            if (SMALL) {                                // v < 68 q < 2^(b + 7)
                v = reduce_small(v, Mc);
            } else {
                v = v >= q2 ? v - q2 : v;
                v = v >= q ? v - q : v;
            }
            sm[swz(off[i])] = v;
        }
        __syncthreads();
        for (int i = tid; i < tile; i += nthr) {
            const uint64_t v = sm[swz(i)];
            const size_t pos = (size_t)blk0 * N2 + i;
            if (EPI) {
                uint64_t r = mul_shoup(sub_mod(ep.u[pos], v, q), ep.pinv.w, ep.pinv.ws, q);
                if (ep.c0) r = add_mod(r, ep.c0[perm_src((uint32_t)pos, ep.g, s1 + s2)], q);
                if (ep.base) r = add_mod(r, ep.base[pos], q);
                ep.o[pos] = r;
            } else {
                a[pos] = v;
            }
        }
    } else if (last) {
#pragma unroll
        for (int i = 0; i < 8; ++i) at[off[i]] = x[i];
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) sm[swz(off[i])] = x[i];
        __syncthreads();
    }
}

// Rounds of a pass of 2^lg points: forward e0 = 0, 3, 6, ...; inverse from the top down.
__device__ __forceinline__ void round_of(int r, int lg, bool inv, int kmax, int& e0, int& K) {
    if (!inv) {
        e0 = kmax * r;
        K = min(kmax, lg - e0);
    } else {
        const int top = lg - kmax * r;
        K = min(kmax, top);
        e0 = top - K;
    }
}

template <bool INV, bool SMALL, int KMAX, bool PRO>
__device__ __forceinline__ void ntt_cols_body(uint64_t* __restrict__ a, uint64_t* sm, int logN,
                                              int s1, int lc, int lo0,
                                              const ShoupPair* __restrict__ w, const ModConst& Mc,
                                              const BConvCta& pc, const ShoupPair& osc) {
    const int N2 = (1 << logN) >> s1;
    const int nr = (s1 + KMAX - 1) / KMAX;
    uint64_t x[8];
    for (int r = 0; r < nr; ++r) {
        int e0, K;
        round_of(r, s1, INV, KMAX, e0, K);
        const bool first = r == 0, last = r == nr - 1;
        if (KMAX == 3 && K == 3) col_round<3, INV, SMALL, PRO>(x, sm, a, first, last, e0, s1, N2, lo0, lc, w, Mc, pc, osc);
        else if (K == 2) col_round<2, INV, SMALL, PRO>(x, sm, a, first, last, e0, s1, N2, lo0, lc, w, Mc, pc, osc);
        else col_round<1, INV, SMALL, PRO>(x, sm, a, first, last, e0, s1, N2, lo0, lc, w, Mc, pc, osc);
    }
}

template <bool INV, bool SMALL, int KMAX, bool EPI>
__device__ __forceinline__ void ntt_rows_body(uint64_t* __restrict__ a, uint64_t* sm, int logN,
                                              int s1, int blk0,
                                              const ShoupPair* __restrict__ w, const ModConst& Mc,
                                              const CombineCta& ep) {
    const int s2 = logN - s1;
    const int nr = (s2 + KMAX - 1) / KMAX;
    uint64_t x[8];
    for (int r = 0; r < nr; ++r) {
        int e0, K;
        round_of(r, s2, INV, KMAX, e0, K);
        const bool first = r == 0, last = r == nr - 1;
        if (KMAX == 3 && K == 3) row_round<3, INV, SMALL, EPI>(x, sm, a, first, last, e0, s1, s2, blk0, w, Mc, ep);
        else if (K == 2) row_round<2, INV, SMALL, EPI>(x, sm, a, first, last, e0, s1, s2, blk0, w, Mc, ep);
        else row_round<1, INV, SMALL, EPI>(x, sm, a, first, last, e0, s1, s2, blk0, w, Mc, ep);
    }
}

// The forward transform of a modulus below 2^57 takes the unreduced butterflies (SMALL, see
// the header); the launcher splits a launch's limbs by that test.
bool small_mod(uint64_t q) { return (q >> 57) == 0; }
// The inverse transform of a modulus below 2^61 keeps its values in [0, 4q) (bfly_gs_small).
bool small_inv_mod(uint64_t q) { return (q >> 61) == 0; }

// Column pass.  Inverse: the last round multiplies by oscale[row] when given, else N^-1.
// Forward with PRO: the first round reads the fused base conversion `bc` instead of `data`.
template <bool INV, bool SMALL, int KMAX, bool PRO>
__global__ void __launch_bounds__(256, 4)
k_ntt_cols(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1, int lc,
           const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw,
           const ShoupPair* __restrict__ oscale, const BConvSrc bc) {
    __shared__ uint64_t sm[kTile];
    __shared__ ShoupPair csm[8];
    const int N = 1 << logN;
    const int mod = mod_off + blockIdx.y;
    const ModConst Mc = mods[mod];
    const ShoupPair* w = tw + (size_t)mod * N;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N;
    const int lo0 = blockIdx.x << lc;
    ShoupPair osc{Mc.n_inv, Mc.n_inv_sh};
    if (INV && oscale) osc = oscale[blockIdx.y];
    BConvCta pc{nullptr, csm, 0, N};
    if (PRO) {
        if ((int)threadIdx.x < bc.ns) csm[threadIdx.x] = bc.cst[(size_t)threadIdx.x * bc.cst_s + mod];
        __syncthreads();
        pc.s = bc.src + blockIdx.z * bc.src_stride;
        pc.ns = bc.ns;
    }
    ntt_cols_body<INV, SMALL, KMAX, PRO>(a, sm, logN, s1, lc, lo0, w, Mc, pc, osc);
}

// Row pass.  Forward with EPI: the last round writes the combine step `cd` instead of v.  The
// unreduced forward rounds hold more live values: three CTAs per SM leave them in registers
// (measured faster than four with spills).
template <bool INV, bool SMALL, int KMAX, bool EPI>
__global__ void __launch_bounds__(256, (SMALL && !INV) ? 3 : 4)
k_ntt_rows(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1, int blocks,
           const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw, const CombineDst cd) {
    __shared__ uint64_t sm[kTile];
    const int N = 1 << logN;
    const int mod = mod_off + blockIdx.y;
    const ModConst Mc = mods[mod];
    const ShoupPair* w = tw + (size_t)mod * N;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N;
    const int blk0 = blockIdx.x * blocks;
    CombineCta ep{nullptr, nullptr, nullptr, nullptr, ShoupPair{0, 0}, 1u};
    if (EPI) {
        const int it = blockIdx.z >> 1, k = blockIdx.z & 1;
        const size_t row = (size_t)k * cd.L * N + (size_t)mod * N;
        ep.u = cd.u + blockIdx.z * cd.u_stride + (size_t)mod * N;
        ep.o = cd.outp[it] + row;
        ep.c0 = (k == 0 && cd.c0p) ? cd.c0p[it] + (size_t)mod * N : nullptr;
        ep.base = cd.basep ? cd.basep[it] + row : nullptr;
        ep.pinv = cd.pinv[mod];
        ep.g = cd.g;
    }
    ntt_rows_body<INV, SMALL, KMAX, EPI>(a, sm, logN, s1, blk0, w, Mc, ep);
}

struct Split {
    int s1, cols, lc, col_ctas, col_threads, blocks, row_ctas, row_threads;
};

// The split N = N1 N2 with the fewest radix-8 rounds (ceil(s1/3) + ceil(s2/3), both passes at
// most kTile points); among those the most balanced, then the smaller N1 (more adjacent columns
// per CTA in the column pass).  A candidate for the autotuner; the default split is
// s1 = floor(log N / 2) (measured faster at N = 2^15 although it takes one more round).
int best_s1(int logN) {
    int best = logN / 2, best_cost = 1 << 30, best_tilt = 1 << 30;
    for (int s = 1; s < logN; ++s) {
        if ((1 << s) > kTile || (1 << (logN - s)) > kTile) continue;
        const int cost = (s + 2) / 3 + (logN - s + 2) / 3;
        const int tilt = 2 * s > logN ? 2 * s - logN : logN - 2 * s;
        if (cost < best_cost || (cost == best_cost && tilt < best_tilt)) {
            best = s;
            best_cost = cost;
            best_tilt = tilt;
        }
    }
    return best;
}

bool split_ok(int logN, int s1) {
    return s1 >= 1 && s1 < logN && (1 << s1) <= kTile && (1 << (logN - s1)) <= kTile;
}

Split split_of(int logN, int s1) {
    Split sp;
    sp.s1 = split_ok(logN, s1) ? s1 : logN / 2;
    const int N1 = 1 << sp.s1, N2 = 1 << (logN - sp.s1);
    sp.cols = kTile / N1;
    if (sp.cols > N2) sp.cols = N2;
    if (sp.cols < 1) sp.cols = 1;
    sp.lc = 0;
    while ((1 << sp.lc) < sp.cols) ++sp.lc;
    sp.col_ctas = N2 / sp.cols;
    sp.col_threads = N1 * sp.cols / 8;
    sp.blocks = kTile / N2;
    if (sp.blocks > N1) sp.blocks = N1;
    if (sp.blocks < 1) sp.blocks = 1;
    sp.row_ctas = N1 / sp.blocks;
    sp.row_threads = sp.blocks * N2 / 8;
    return sp;
}

}  // namespace

int ntt_split_candidates(int logN, int* out, int cap) {
    int n = 0;
    const int cand[4] = {logN / 2, best_s1(logN), logN / 2 - 1, logN / 2 + 1};
    for (int c : cand) {
        if (!split_ok(logN, c)) continue;
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= out[i] == c;
        if (!dup && n < cap) out[n++] = c;
    }
    return n;
}

namespace {

// Forward row table from the standard one: entry e of stage s >= s1 (offset o = e - 2^s,
// o = base 2^ee + j with ee = (s - s1) mod kmax, the stage's place in its round) moves to
// 2^s + j 2^(s - ee) + base; stages below s1 are copied.
__global__ void k_row_table(const ShoupPair* __restrict__ fwd, ShoupPair* __restrict__ fwd_r,
                            int logN, int s1, int kmax, size_t total) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t N = (size_t)1 << logN, base_m = i - (i & (N - 1));
    const int e = (int)(i & (N - 1));
    if (e < (1 << s1)) {
        fwd_r[i] = fwd[i];
        return;
    }
    const int s = 31 - __clz(e), o = e - (1 << s), ee = (s - s1) % kmax;
    const int b = o >> ee, j = o & ((1 << ee) - 1);
    fwd_r[base_m + (1 << s) + ((size_t)j << (s - ee)) + b] = fwd[i];
}

// Rebuilds the row table for a split and radix cap it was not made for.  ntt_prepare does
// it wherever those change; a transform that still finds them stale rebuilds them, except
// while recording (the rebuild would enter the graph), where the recording is spoiled.
void ensure_row_tables(he_ctx* ctx, int s1, int kmax) {
    if (ctx->tw_rows_s1 == s1 && ctx->tw_rows_k == kmax) return;
    if (ctx->rec) {
        he_fail(ctx, HE_EINVAL, "NTT twiddle order changed while recording");
        return;
    }
    const size_t total = (size_t)ctx->n_mod * ctx->N;
    ++ctx->launches;
    k_row_table<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_tw_fwd, ctx->d_tw_fwd_rows, ctx->logN, s1, kmax, total);
    ctx->tw_rows_s1 = s1;
    ctx->tw_rows_k = kmax;
}

}  // namespace

void ntt_prepare(he_ctx* ctx) {
    const Split sp = split_of(ctx->logN, ctx->ntt_s1);
    ensure_row_tables(ctx, sp.s1, ctx->ntt_radix == 2 ? 2 : 3);
}

constexpr CombineDst kNoCombine{nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0, 1u};

template <bool INV, bool SMALL, int KMAX, bool PRO = false, bool EPI = false>
void launch_pass_pair(he_ctx* ctx, const Split& sp, uint64_t* d, int items, size_t item_stride,
                      int rows, int mod, const ShoupPair* oscale = nullptr,
                      const BConvSrc& bc = BConvSrc{nullptr, 0, nullptr, 0, 0},
                      const CombineDst& cd = kNoCombine) {
    dim3 gc(sp.col_ctas, rows, items), gr(sp.row_ctas, rows, items);
    ensure_row_tables(ctx, sp.s1, KMAX);
    ctx->launches += 2;
    const ShoupPair* tw = INV ? ctx->d_tw_inv : ctx->d_tw_fwd;
    const ShoupPair* twr = INV ? ctx->d_tw_inv : ctx->d_tw_fwd_rows;
    if (!INV) {
        k_ntt_cols<INV, SMALL, KMAX, PRO><<<gc, sp.col_threads, 0, ctx->stream>>>(
            d, item_stride, mod, ctx->logN, sp.s1, sp.lc, ctx->d_mod, tw, nullptr, bc);
        k_ntt_rows<INV, SMALL, KMAX, EPI><<<gr, sp.row_threads, 0, ctx->stream>>>(
            d, item_stride, mod, ctx->logN, sp.s1, sp.blocks, ctx->d_mod, twr, cd);
    } else {
        k_ntt_rows<INV, SMALL, KMAX, false><<<gr, sp.row_threads, 0, ctx->stream>>>(
            d, item_stride, mod, ctx->logN, sp.s1, sp.blocks, ctx->d_mod, twr, kNoCombine);
        k_ntt_cols<INV, SMALL, KMAX, false><<<gc, sp.col_threads, 0, ctx->stream>>>(
            d, item_stride, mod, ctx->logN, sp.s1, sp.lc, ctx->d_mod, tw, oscale, bc);
    }
}

template <bool PRO, bool EPI = false>
static void forward_runs(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                         int mod_off, const BConvSrc& bc, const CombineDst& cd = kNoCombine) {
    if (items <= 0 || rows <= 0) return;
    const Split sp = split_of(ctx->logN, ctx->ntt_s1);
    const bool r4 = ctx->ntt_radix == 2;
    // runs of limbs of one kind (moduli below 2^57 or not), one launch pair each
    for (int r0 = 0; r0 < rows;) {
        const bool small = small_mod(ctx->mods[mod_off + r0]);
        int r1 = r0 + 1;
        while (r1 < rows && small_mod(ctx->mods[mod_off + r1]) == small) ++r1;
        uint64_t* d = data + (size_t)r0 * ctx->N;
        const int n = r1 - r0, m = mod_off + r0;
        if (small) {
            if (r4) launch_pass_pair<false, true, 2, PRO, EPI>(ctx, sp, d, items, item_stride, n, m, nullptr, bc, cd);
            else launch_pass_pair<false, true, 3, PRO, EPI>(ctx, sp, d, items, item_stride, n, m, nullptr, bc, cd);
        } else {
            if (r4) launch_pass_pair<false, false, 2, PRO, EPI>(ctx, sp, d, items, item_stride, n, m, nullptr, bc, cd);
            else launch_pass_pair<false, false, 3, PRO, EPI>(ctx, sp, d, items, item_stride, n, m, nullptr, bc, cd);
        }
        r0 = r1;
    }
}

void ntt_forward(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off) {
    forward_runs<false>(ctx, data, items, item_stride, rows, mod_off,
                        BConvSrc{nullptr, 0, nullptr, 0, 0});
}

void ntt_forward_bconv(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                       int mod_off, const BConvSrc& bc) {
    forward_runs<true>(ctx, data, items, item_stride, rows, mod_off, bc);
}

void ntt_forward_bconv_combine(he_ctx* ctx, uint64_t* data, int items, size_t item_stride,
                               int rows, const BConvSrc& bc, const CombineDst& cd) {
    forward_runs<true, true>(ctx, data, items, item_stride, rows, 0, bc, cd);
}

void ntt_inverse_scaled(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                        int mod_off, const ShoupPair* scale) {
    if (items <= 0 || rows <= 0) return;
    const Split sp = split_of(ctx->logN, ctx->ntt_s1);
    const bool r4 = ctx->ntt_radix == 2;
    for (int r0 = 0; r0 < rows;) {                   // runs of limbs of one kind
        const bool small = small_inv_mod(ctx->mods[mod_off + r0]);
        int r1 = r0 + 1;
        while (r1 < rows && small_inv_mod(ctx->mods[mod_off + r1]) == small) ++r1;
        uint64_t* d = data + (size_t)r0 * ctx->N;
        const int n = r1 - r0, m = mod_off + r0;
        const ShoupPair* sc = scale ? scale + r0 : nullptr;
        if (small) {
            if (r4) launch_pass_pair<true, true, 2>(ctx, sp, d, items, item_stride, n, m, sc);
            else launch_pass_pair<true, true, 3>(ctx, sp, d, items, item_stride, n, m, sc);
        } else {
            if (r4) launch_pass_pair<true, false, 2>(ctx, sp, d, items, item_stride, n, m, sc);
            else launch_pass_pair<true, false, 3>(ctx, sp, d, items, item_stride, n, m, sc);
        }
        r0 = r1;
    }
}

void ntt_inverse(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off) {
    ntt_inverse_scaled(ctx, data, items, item_stride, rows, mod_off, nullptr);
}
