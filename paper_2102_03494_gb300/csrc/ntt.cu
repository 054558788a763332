// ntt.cu -- negacyclic NTT / inverse NTT over Z_q[X]/(X^N+1), batched over limbs and items.
//
// Forward transform: merged-psi Cooley-Tukey, stage s (m = 2^s, t = N / 2^(s+1)) pairs
// (j, j+t) in group i = j / 2t with twiddle psi^brv(m + i); the output is in bit-reversed
// order, position p holding a(psi^(2 brv(p) + 1)).  Inverse: Gentleman-Sande with
// psi^-brv(m + i), stages in reverse, then the factor N^-1.
//
// The N = N1 N2 points (N1 = 2^s1, s1 = floor(log N / 2)) are split in two passes, each
// staged in shared memory:
//   column pass: stages s < s1 act on elements with the same j mod N2 (strided columns);
//                one CTA holds COLS adjacent columns x N1 rows (128-byte row segments);
//   row pass:    stages s >= s1 act inside contiguous blocks of N2 elements; one CTA holds
//                several blocks.
// Each pass reads and writes every limb once.
#include "he_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTileElems = 2048;   // elements staged per CTA (16 KiB)

__global__ void __launch_bounds__(kThreads)
k_fwd_cols(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1,
           int cols, const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw) {
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, N1 = 1 << s1, N2 = N >> s1;
    const int mod = mod_off + blockIdx.y;
    const uint64_t q = mods[mod].q;
    const ShoupPair* w = tw + (size_t)mod * N;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N;
    const int lo0 = blockIdx.x * cols;
    const int total = N1 * cols;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int hi = idx / cols, c = idx - hi * cols;
        sm[idx] = a[(size_t)hi * N2 + lo0 + c];
    }
    __syncthreads();
    const int nb = total >> 1;
    for (int s = 0; s < s1; ++s) {
        const int tt = N1 >> (s + 1);
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int bb = b / cols, c = b - bb * cols;
            int grp = bb / tt;
            int rj = grp * 2 * tt + (bb - grp * tt);
            ShoupPair W = w[(1 << s) + grp];
            uint64_t* pu = sm + rj * cols + c;
            uint64_t* pv = pu + tt * cols;
            uint64_t U = *pu;
            uint64_t V = mul_shoup(*pv, W.w, W.ws, q);
            *pu = add_mod(U, V, q);
            *pv = sub_mod(U, V, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int hi = idx / cols, c = idx - hi * cols;
        a[(size_t)hi * N2 + lo0 + c] = sm[idx];
    }
}

__global__ void __launch_bounds__(kThreads)
k_fwd_rows(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1,
           int blocks, const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw) {
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, N2 = N >> s1;
    const int mod = mod_off + blockIdx.y;
    const uint64_t q = mods[mod].q;
    const ShoupPair* w = tw + (size_t)mod * N;
    const int hi0 = blockIdx.x * blocks;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N + (size_t)hi0 * N2;
    const int total = blocks * N2;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    const int half = N2 >> 1, nb = total >> 1;
    for (int s = s1; s < logN; ++s) {
        const int tl = N2 >> (s - s1 + 1);
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int g = b / half, lb = b - g * half;
            int grp = lb / tl;
            int lj = grp * 2 * tl + (lb - grp * tl);
            ShoupPair W = w[(1 << s) + ((hi0 + g) << (s - s1)) + grp];
            uint64_t* pu = sm + g * N2 + lj;
            uint64_t* pv = pu + tl;
            uint64_t U = *pu;
            uint64_t V = mul_shoup(*pv, W.w, W.ws, q);
            *pu = add_mod(U, V, q);
            *pv = sub_mod(U, V, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) a[idx] = sm[idx];
}

__global__ void __launch_bounds__(kThreads)
k_inv_rows(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1,
           int blocks, const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw) {
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, N2 = N >> s1;
    const int mod = mod_off + blockIdx.y;
    const uint64_t q = mods[mod].q;
    const ShoupPair* w = tw + (size_t)mod * N;
    const int hi0 = blockIdx.x * blocks;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N + (size_t)hi0 * N2;
    const int total = blocks * N2;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    const int half = N2 >> 1, nb = total >> 1;
    for (int s = logN - 1; s >= s1; --s) {
        const int tl = N2 >> (s - s1 + 1);
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int g = b / half, lb = b - g * half;
            int grp = lb / tl;
            int lj = grp * 2 * tl + (lb - grp * tl);
            ShoupPair W = w[(1 << s) + ((hi0 + g) << (s - s1)) + grp];
            uint64_t* pu = sm + g * N2 + lj;
            uint64_t* pv = pu + tl;
            uint64_t U = *pu, V = *pv;
            *pu = add_mod(U, V, q);
            *pv = mul_shoup(sub_mod(U, V, q), W.w, W.ws, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) a[idx] = sm[idx];
}

__global__ void __launch_bounds__(kThreads)
k_inv_cols(uint64_t* __restrict__ data, size_t item_stride, int mod_off, int logN, int s1,
           int cols, const ModConst* __restrict__ mods, const ShoupPair* __restrict__ tw) {
    extern __shared__ uint64_t sm[];
    const int N = 1 << logN, N1 = 1 << s1, N2 = N >> s1;
    const int mod = mod_off + blockIdx.y;
    const ModConst M = mods[mod];
    const uint64_t q = M.q;
    const ShoupPair* w = tw + (size_t)mod * N;
    uint64_t* a = data + blockIdx.z * item_stride + (size_t)blockIdx.y * N;
    const int lo0 = blockIdx.x * cols;
    const int total = N1 * cols;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int hi = idx / cols, c = idx - hi * cols;
        sm[idx] = a[(size_t)hi * N2 + lo0 + c];
    }
    __syncthreads();
    const int nb = total >> 1;
    for (int s = s1 - 1; s >= 0; --s) {
        const int tt = N1 >> (s + 1);
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int bb = b / cols, c = b - bb * cols;
            int grp = bb / tt;
            int rj = grp * 2 * tt + (bb - grp * tt);
            ShoupPair W = w[(1 << s) + grp];
            uint64_t* pu = sm + rj * cols + c;
            uint64_t* pv = pu + tt * cols;
            uint64_t U = *pu, V = *pv;
            *pu = add_mod(U, V, q);
            *pv = mul_shoup(sub_mod(U, V, q), W.w, W.ws, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int hi = idx / cols, c = idx - hi * cols;
        a[(size_t)hi * N2 + lo0 + c] = mul_shoup(sm[idx], M.n_inv, M.n_inv_sh, q);
    }
}

struct Split {
    int s1, cols, col_ctas, blocks, row_ctas;
};

Split split_of(int logN) {
    Split sp;
    sp.s1 = logN / 2;
    int N1 = 1 << sp.s1, N2 = 1 << (logN - sp.s1);
    sp.cols = N2 < 16 ? N2 : 16;
    while (sp.cols > 1 && N1 * sp.cols > kTileElems) sp.cols >>= 1;
    sp.col_ctas = N2 / sp.cols;
    sp.blocks = kTileElems / N2;
    if (sp.blocks < 1) sp.blocks = 1;
    if (sp.blocks > N1) sp.blocks = N1;
    sp.row_ctas = N1 / sp.blocks;
    return sp;
}

int block_threads(int elems) {
    int t = elems / 2;
    if (t > kThreads) t = kThreads;
    if (t < 32) t = 32;
    return t;
}

}  // namespace

void ntt_forward(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off) {
    if (items <= 0 || rows <= 0) return;
    ctx->launches += 2;
    Split sp = split_of(ctx->logN);
    int N1 = 1 << sp.s1, N2 = ctx->N >> sp.s1;
    dim3 gc(sp.col_ctas, rows, items), gr(sp.row_ctas, rows, items);
    size_t smc = (size_t)N1 * sp.cols * 8, smr = (size_t)sp.blocks * N2 * 8;
    k_fwd_cols<<<gc, block_threads(N1 * sp.cols), smc, ctx->stream>>>(
        data, item_stride, mod_off, ctx->logN, sp.s1, sp.cols, ctx->d_mod, ctx->d_tw_fwd);
    k_fwd_rows<<<gr, block_threads(sp.blocks * N2), smr, ctx->stream>>>(
        data, item_stride, mod_off, ctx->logN, sp.s1, sp.blocks, ctx->d_mod, ctx->d_tw_fwd);
}

void ntt_inverse(he_ctx* ctx, uint64_t* data, int items, size_t item_stride, int rows,
                 int mod_off) {
    if (items <= 0 || rows <= 0) return;
    ctx->launches += 2;
    Split sp = split_of(ctx->logN);
    int N1 = 1 << sp.s1, N2 = ctx->N >> sp.s1;
    dim3 gc(sp.col_ctas, rows, items), gr(sp.row_ctas, rows, items);
    size_t smc = (size_t)N1 * sp.cols * 8, smr = (size_t)sp.blocks * N2 * 8;
    k_inv_rows<<<gr, block_threads(sp.blocks * N2), smr, ctx->stream>>>(
        data, item_stride, mod_off, ctx->logN, sp.s1, sp.blocks, ctx->d_mod, ctx->d_tw_inv);
    k_inv_cols<<<gc, block_threads(N1 * sp.cols), smc, ctx->stream>>>(
        data, item_stride, mod_off, ctx->logN, sp.s1, sp.cols, ctx->d_mod, ctx->d_tw_inv);
}
