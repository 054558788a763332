// deepnet.cu -- convolution layers over several ciphertexts per tensor, and the deeper network
// built from them (stride-1 "same" convolutions, factorized or not, x^2, global sum pooling
// and a fully connected classifier, the last two evaluated as one linear map).
//
// Tensor layout: channel c of an H x W map occupies block c mod g of ciphertext c / g (row 0),
// block size Bk = next_pow2(H W), g = (N/2) / Bk, pixel (h, w) at offset h W + w.
//
// Layer: for every input ciphertext the d^2 taps are rotations by delta = (i - pad) W +
// (j - pad), hoisted and left in Q u P; the fused tap kernel sums, for each low-rank channel c',
// the tap products of all input ciphertexts of an image (per-tap input selection) and one
// ModDown follows.  The block sum y1[c'] = sum_{u<g} rot(acc, u Bk) -- its g - 1 rotations
// hoisted from one ModUp and summed in Q u P by the same tap kernel against the plaintext 1,
// one ModDown -- leaves the channel replicated in every block, so the restore needs no
// rotation: output ciphertext
// G is sum_c' y1[c'] * P[G][c'], P[G][c'] holding W2[G g + j][c'] on the pixels of block j
// (for the unfactorized layer W2 is the identity and r = O_c).
#include <algorithm>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

namespace {

int next_pow2_i(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

int ilog2(int x) {
    int k = 0;
    while ((1 << k) < x) ++k;
    return k;
}

// Tap plaintext slots for channels [c0, c0 + cn) and taps [t0, t0 + nt) of the layer, tap
// t = gi d^2 + i d + j (input ciphertext gi): slots[(c nt + u) N + p] = W1[c0 + c][ci][i][j] at
// the output pixel p of block b (channel ci = gi g + b) whose input pixel lies in the image.
__global__ void k_mc_tap_slots(const int32_t* __restrict__ W1, int C_in, int H, int W, int d,
                               int pad, int lbk, int g, int c0, int nt, int t0, int logN,
                               int64_t* __restrict__ slots) {
    const int N = 1 << logN;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int c = blockIdx.y / nt, u = blockIdx.y - c * nt;
    const int t = t0 + u, dd = d * d;
    const int gi = t / dd, ij = t - gi * dd, i = ij / d, j = ij - i * d;
    int64_t v = 0;
    if (p < N / 2) {
        const int b = p >> lbk, off = p & ((1 << lbk) - 1);
        const int ci = gi * g + b;
        if (ci < C_in && off < H * W) {
            const int oh = off / W, ow = off - oh * W;
            const int h = oh + i - pad, w = ow + j - pad;
            if (h >= 0 && h < H && w >= 0 && w < W)
                v = W1[(((size_t)(c0 + c) * C_in + ci) * d + i) * d + j];
        }
    }
    slots[(size_t)blockIdx.y * N + p] = v;
}

// Restore plaintext slots P[G][c] for G < n_out and channels [c0, c0 + cn):
// W2[G g + b][c0 + c] on the pixels of block b (the identity when W2 is null).
__global__ void k_mc_restore_slots(const int32_t* __restrict__ W2, int r, int O_c, int H, int W,
                                   int lbk, int g, int c0, int cn, int logN,
                                   int64_t* __restrict__ slots) {
    const int N = 1 << logN;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int G = blockIdx.y / cn, c = blockIdx.y - G * cn;
    int64_t v = 0;
    if (p < N / 2) {
        const int b = p >> lbk, off = p & ((1 << lbk) - 1);
        const int o = G * g + b;
        if (o < O_c && off < H * W)
            v = W2 ? W2[(size_t)o * r + c0 + c] : (o == c0 + c ? 1 : 0);
    }
    slots[(size_t)blockIdx.y * N + p] = v;
}

// copies[t][l][n] = 2^64 mod q_l (the plaintext 1 in Montgomery form), t < copies, l < rows.
__global__ void k_mont_ones(uint64_t* __restrict__ out, int rows, int copies, int logN,
                            const ModConst* __restrict__ mods) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    const uint64_t one = to_mont(1, mods[l]);
    for (int t = 0; t < copies; ++t) out[((size_t)t * rows + l) * N + n] = one;
}

struct McGeom {
    int Bk, lbk, g, n_in, n_out, r, taps, T;
};

int mc_geom(he_ctx* ctx, const he_mc_conv* cv, McGeom* m) {
    if (!cv || cv->C_in < 1 || cv->H < 1 || cv->W < 1 || cv->d < 1 || cv->pad < 0 ||
        cv->d != 2 * cv->pad + 1 || cv->O_c < 1 || cv->r < 0)
        return he_fail(ctx, HE_EINVAL, "he_mc_conv: shape out of range (odd d, pad = (d - 1) / 2)");
    m->Bk = next_pow2_i(cv->H * cv->W);
    m->lbk = ilog2(m->Bk);
    m->g = (ctx->N / 2) / m->Bk;
    if (m->g < 1) return he_fail(ctx, HE_EINVAL, "he_mc_conv: one channel map must fit in a row");
    m->n_in = (cv->C_in + m->g - 1) / m->g;
    m->n_out = (cv->O_c + m->g - 1) / m->g;
    m->r = cv->r ? cv->r : cv->O_c;
    m->taps = cv->d * cv->d;
    m->T = m->n_in * m->taps;
    if (m->n_in > 255) return he_fail(ctx, HE_EINVAL, "he_mc_conv: too many input ciphertexts");
    return HE_OK;
}

std::vector<int32_t> mc_conv_steps(const he_mc_conv& cv, const McGeom& m) {
    std::vector<int32_t> st;
    for (int i = 0; i < cv.d; ++i)
        for (int j = 0; j < cv.d; ++j) {
            const int dl = (i - cv.pad) * cv.W + (j - cv.pad);
            if (dl) st.push_back(dl);
        }
    for (int u = 1; u < m.g; ++u) st.push_back(u * m.Bk);
    return st;
}

}  // namespace

extern "C" int he_mc_conv_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* lowrank_w,
                                const int32_t* restore_w, const he_mc_conv* conv, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!in || !lowrank_w || !out || B < 1) return he_fail(ctx, HE_EINVAL, "he_mc_conv: null argument");
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_mc_conv: t is not 1 mod 2N");
    McGeom m;
    int rc = mc_geom(ctx, conv, &m);
    if (rc) return rc;
    if ((conv->r == 0) != (restore_w == nullptr))
        return he_fail(ctx, HE_EINVAL, "he_mc_conv: restore weights go with r > 0 only");
    const int L = ctx->L, LK = L + ctx->K;
    for (int i = 0; i < B * m.n_in; ++i)
        if ((rc = check_ct(ctx, &in[i], L, HE_NTT, "he_mc_conv input"))) return rc;
    for (int i = 0; i < B * m.n_out; ++i)
        if ((rc = check_ct(ctx, &out[i], L, -1, "he_mc_conv output"))) return rc;
    // keys: tap offsets then fold steps
    std::vector<uint32_t> tap_g(m.taps, 1u);
    std::vector<const uint64_t*> tap_key(m.taps, nullptr);
    for (int i = 0; i < conv->d; ++i)
        for (int j = 0; j < conv->d; ++j) {
            const int dl = (i - conv->pad) * conv->W + (j - conv->pad);
            if (!dl) continue;
            tap_g[i * conv->d + j] = galois_elt(ctx, dl);
            if ((rc = he_get_key(ctx, tap_g[i * conv->d + j], &tap_key[i * conv->d + j]))) return rc;
        }
    // block sum: rotations by u Bk, u = 1 .. g - 1 (tap u of the block-sum tap table)
    std::vector<uint32_t> fold_g;
    std::vector<const uint64_t*> fold_key;
    for (int u = 1; u < m.g; ++u) {
        fold_g.push_back(galois_elt(ctx, u * m.Bk));
        fold_key.push_back(nullptr);
        if ((rc = he_get_key(ctx, fold_g.back(), &fold_key.back()))) return rc;
    }
    if (m.g > HE_MAX_TAPS) return he_fail(ctx, HE_EINVAL, "he_mc_conv: too many blocks per row");
    const size_t N = ctx->N, ct = 2 * (size_t)L * N, ext_ct = 2 * (size_t)LK * N;
    const size_t items = (size_t)B * m.n_in;
    const int CH = std::min(m.r, 8);                         // low-rank channels per pass
    const int tmax = std::min(m.T, HE_MAX_TAPS);             // taps per tap launch
    const int n_tc = (m.T + tmax - 1) / tmax;
    const int fold_items = B * CH;                           // ciphertexts block-summed at once
    const size_t w1n = (size_t)m.r * conv->C_in * m.taps, w2n = restore_w ? (size_t)conv->O_c * m.r : 0;
    const size_t need = items * ct * 2                            // X, P x
                        + items * rot_scratch_per_item(ctx)       // input ModUp digits
                        + (size_t)fold_items * rot_scratch_per_item(ctx)
                        + (size_t)fold_items * (ct + ext_ct)      // P y1, block sums
                        + (size_t)m.g * LK * N                    // the plaintext 1
                        + (size_t)CH * tmax * (2 * N + (size_t)LK * N)   // tap slots, tmp, plaintexts
                        + (size_t)B * CH * ext_ct * (n_tc > 1 ? 2 : 1)
                        + (size_t)B * CH * ct * 3                 // y1, its fold partner, ModDown
                        + (size_t)m.n_out * CH * (2 * N + (size_t)L * N)  // restore plaintexts
                        + (w1n + w2n) / 2 + 2 + 32 * 24;
    if ((rc = arena_reserve(ctx, need))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, items * ct);
    uint64_t* XP = arena_take(ctx, items * ct);
    RotBufs rb = rot_bufs_take(ctx, (int)items);
    RotBufs rbf = rot_bufs_take(ctx, fold_items);
    uint64_t* YP = arena_take(ctx, (size_t)fold_items * ct);
    uint64_t* AF = arena_take(ctx, (size_t)fold_items * ext_ct);
    uint64_t* ones = arena_take(ctx, (size_t)m.g * LK * N);
    int64_t* slots = (int64_t*)arena_take(ctx, (size_t)CH * tmax * N);
    uint64_t* tmp = arena_take(ctx, (size_t)CH * tmax * N);
    uint64_t* pts = arena_take(ctx, (size_t)CH * tmax * LK * N);
    uint64_t* AX = arena_take(ctx, (size_t)B * CH * ext_ct);
    uint64_t* AX2 = n_tc > 1 ? arena_take(ctx, (size_t)B * CH * ext_ct) : nullptr;
    uint64_t* Y = arena_take(ctx, (size_t)B * CH * ct);
    uint64_t* Y2 = arena_take(ctx, (size_t)B * CH * ct);
    uint64_t* V = arena_take(ctx, (size_t)B * CH * ct);
    int64_t* rslots = (int64_t*)arena_take(ctx, (size_t)m.n_out * CH * N);
    uint64_t* rtmp = arena_take(ctx, (size_t)m.n_out * CH * N);
    uint64_t* rpts = arena_take(ctx, (size_t)m.n_out * CH * L * N);
    int32_t* d_w1 = (int32_t*)arena_take(ctx, (w1n + 1) / 2);
    int32_t* d_w2 = w2n ? (int32_t*)arena_take(ctx, (w2n + 1) / 2) : nullptr;
    if (!d_w1 || !rb.v || !rbf.v || !ones) return he_fail(ctx, HE_ENOMEM, "he_mc_conv: scratch");
    ++ctx->launches;
    k_mont_ones<<<dim3((unsigned)((N + 255) / 256), LK), 256, 0, ctx->stream>>>(ones, LK, m.g,
                                                                            ctx->logN, ctx->d_mod);

    if ((rc = upload_host(ctx, d_w1, lowrank_w, w1n * 4))) return rc;
    if (w2n && (rc = upload_host(ctx, d_w2, restore_w, w2n * 4))) return rc;
    for (size_t i = 0; i < items; ++i)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + i * ct, in[i].data, ct * 8, cudaMemcpyDeviceToDevice,
                                           ctx->stream));
    phase_begin(ctx, HE_PHASE_MODUP);
    modup_items(ctx, X, (int)items, 1u, rb);
    launch_scale_p(ctx, X, XP, (int)items);
    phase_end(ctx);

    uint64_t nz_restore = 0;
    for (int c0 = 0; c0 < m.r; c0 += CH) {
        const int cn = std::min(CH, m.r - c0);
        // W1 taps of channels [c0, c0 + cn) over every input ciphertext, summed in Q u P
        for (int tc = 0; tc < n_tc; ++tc) {
            const int t0 = tc * tmax, nt = std::min(tmax, m.T - t0);
            phase_begin(ctx, HE_PHASE_ENCODE);
            ++ctx->launches;
            k_mc_tap_slots<<<dim3((unsigned)((N + 255) / 256), cn * nt), 256, 0, ctx->stream>>>(
                d_w1, conv->C_in, conv->H, conv->W, conv->d, conv->pad, m.lbk, m.g, c0, nt, t0,
                ctx->logN, slots);
            encode_device(ctx, slots, cn * nt, tmp, pts, 1, LK);
            phase_end(ctx);
            TapTable tt{};
            tt.n = nt;
            tt.r = cn;
            tt.n_sub = m.n_in;
            for (int u = 0; u < nt; ++u) {
                const int t = t0 + u, gi = t / m.taps, ij = t - gi * m.taps;
                tt.key[u] = tap_key[ij];
                tt.g[u] = tap_g[ij];
                tt.sub[u] = (uint8_t)gi;
            }
            phase_begin(ctx, HE_PHASE_TAPS);
            launch_ks_mac_ext(ctx, rb.D, XP, pts, tt, tc ? AX2 : AX, B);
            if (tc) {
                std::vector<const uint64_t*> xa(B * cn), xb(B * cn);
                std::vector<uint64_t*> xo(B * cn);
                for (int q = 0; q < B * cn; ++q) {
                    xa[q] = AX + (size_t)q * ext_ct;
                    xb[q] = AX2 + (size_t)q * ext_ct;
                    xo[q] = AX + (size_t)q * ext_ct;
                }
                auto pa = upload_ptrs(ctx, xa);
                auto pb = upload_ptrs(ctx, xb);
                auto po = upload_out_ptrs(ctx, xo);
                if (!pa || !pb || !po) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
                launch_add_rows(ctx, pa, pb, po, B * cn, LK);
            }
            phase_end(ctx);
        }
        // one ModDown per (image, channel): AX [B][cn][2][LK][N] -> Y [B][cn][2][L][N]
        const int it = B * cn;
        phase_begin(ctx, HE_PHASE_MODDOWN);
        {
            std::vector<uint64_t*> yo(it);
            for (int q = 0; q < it; ++q) yo[q] = Y + (size_t)q * ct;
            auto op = upload_out_ptrs(ctx, yo);
            if (!op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
            moddown_combine(ctx, AX, V, it, nullptr, nullptr, op, 1u);
        }
        phase_end(ctx);
        // block sum: y1 = sum_{u<g} rot(Y, u Bk) (hoisted, summed in Q u P, one ModDown)
        uint64_t* Ya = Y;
        if (m.g > 1) {
            phase_begin(ctx, HE_PHASE_ROTATE);
            modup_items(ctx, Y, it, 1u, rbf);
            launch_scale_p(ctx, Y, YP, it);
            TapTable ft{};
            ft.n = m.g;
            ft.r = 1;
            ft.n_sub = 1;
            for (int u = 0; u < m.g; ++u) {
                ft.key[u] = u ? fold_key[u - 1] : nullptr;
                ft.g[u] = u ? fold_g[u - 1] : 1u;
            }
            launch_ks_mac_ext(ctx, rbf.D, YP, ones, ft, AF, it);
            std::vector<uint64_t*> yo(it);
            for (int q = 0; q < it; ++q) yo[q] = Y2 + (size_t)q * ct;
            auto op = upload_out_ptrs(ctx, yo);
            if (!op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
            moddown_combine(ctx, AF, V, it, nullptr, nullptr, op, 1u);
            Ya = Y2;
            phase_end(ctx);
        }
        // restore: out[b][G] (+)= sum_c y1[b][c] * P[G][c]
        phase_begin(ctx, HE_PHASE_RESTORE);
        ++ctx->launches;
        k_mc_restore_slots<<<dim3((unsigned)((N + 255) / 256), m.n_out * cn), 256, 0, ctx->stream>>>(
            d_w2, m.r, conv->O_c, conv->H, conv->W, m.lbk, m.g, c0, cn, ctx->logN, rslots);
        encode_device(ctx, rslots, m.n_out * cn, rtmp, rpts, 1, L);
        std::vector<const uint64_t*> mx((size_t)B * m.n_out * cn), mp((size_t)B * m.n_out * cn), ai;
        std::vector<uint64_t*> ao((size_t)B * m.n_out);
        for (int b = 0; b < B; ++b)
            for (int G = 0; G < m.n_out; ++G) {
                const size_t q = (size_t)b * m.n_out + G;
                for (int c = 0; c < cn; ++c) {
                    mx[q * cn + c] = Ya + ((size_t)b * cn + c) * ct;
                    mp[q * cn + c] = rpts + ((size_t)G * cn + c) * L * N;
                }
                ao[q] = out[q].data;
                ai.push_back(c0 ? out[q].data : nullptr);
            }
        for (int G = 0; G < m.n_out; ++G)
            for (int c = 0; c < cn; ++c) {
                const int lo = G * m.g, hi = std::min(conv->O_c, lo + m.g);
                if (restore_w || (c0 + c >= lo && c0 + c < hi)) nz_restore += hi - lo > 0 ? 1 : 0;
            }
        auto a1 = upload_ptrs(ctx, mx);
        auto a2 = upload_ptrs(ctx, mp);
        auto a3 = c0 ? upload_ptrs(ctx, ai) : nullptr;
        auto a4 = upload_out_ptrs(ctx, ao);
        if (!a1 || !a2 || !a4 || (c0 && !a3)) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        launch_mac(ctx, a1, a2, cn, a3, a4, B * m.n_out, L);
        phase_end(ctx);
    }
    // MulPC: tap products and nonzero restore products; AddCC: their sums and the block sums;
    // rotations (all hoisted): the taps and the block sums
    const uint64_t rot = (uint64_t)m.n_in * (m.taps - 1) + (uint64_t)m.r * (m.g - 1);
    ctx->ops[0] += (uint64_t)B * ((uint64_t)m.r * m.T + nz_restore);
    ctx->ops[1] += (uint64_t)B * ((uint64_t)m.r * (m.T - 1 + m.g - 1) +
                                  (nz_restore > (uint64_t)m.n_out ? nz_restore - m.n_out : 0));
    ctx->ops[2] += (uint64_t)B * rot;
    ctx->ops[3] += (uint64_t)B * rot;
    for (int i = 0; i < B * m.n_out; ++i) out[i].domain = HE_NTT;
    return he_launch_check(ctx, "he_mc_conv");
}

extern "C" int he_rotate_sum_batch(he_ctx* ctx, he_ct* cts, int n, const int32_t* steps,
                                   int n_steps) {
    if (!ctx) return HE_EINVAL;
    if (!cts || n < 1 || n_steps < 0 || (n_steps && !steps))
        return he_fail(ctx, HE_EINVAL, "he_rotate_sum: null or empty argument");
    int rc;
    const int L = ctx->L;
    for (int i = 0; i < n; ++i)
        if ((rc = check_ct(ctx, &cts[i], L, HE_NTT, "he_rotate_sum"))) return rc;
    std::vector<uint32_t> gs(n_steps);
    for (int s = 0; s < n_steps; ++s) {
        gs[s] = galois_elt(ctx, steps[s]);
        const uint64_t* k = nullptr;
        if ((rc = he_get_key(ctx, gs[s], &k))) return rc;
    }
    if (!n_steps) return HE_OK;
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    const int chunk = std::min(n, 32);
    if ((rc = arena_reserve(ctx, (size_t)n * ct * 2 + (size_t)chunk * rot_scratch_per_item(ctx) + 32 * 8)))
        return rc;
    arena_reset(ctx);
    uint64_t* A = arena_take(ctx, (size_t)n * ct);
    uint64_t* A2 = arena_take(ctx, (size_t)n * ct);
    RotBufs rb = rot_bufs_take(ctx, chunk);
    if (!rb.v) return he_fail(ctx, HE_ENOMEM, "he_rotate_sum: scratch");
    for (int i = 0; i < n; ++i)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(A + (size_t)i * ct, cts[i].data, ct * 8,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    phase_begin(ctx, HE_PHASE_ROTATE);
    for (int s = 0; s < n_steps; ++s) {
        std::vector<uint64_t*> o(n);
        for (int i = 0; i < n; ++i) o[i] = s == n_steps - 1 ? cts[i].data : A2 + (size_t)i * ct;
        if ((rc = rotate_contig(ctx, A, n, gs[s], A, o, rb, chunk))) return rc;
        std::swap(A, A2);
    }
    phase_end(ctx);
    return he_launch_check(ctx, "he_rotate_sum");
}

extern "C" int he_deep_required_steps(const he_ctx* ctx, const he_mc_conv* convs, int n_layers,
                                      int n_cls, int32_t* steps_out, int cap) {
    if (!ctx || !convs || n_layers < 1 || n_cls < 1) return HE_EINVAL;
    he_ctx* c = const_cast<he_ctx*>(ctx);
    const int half = ctx->N / 2;
    std::vector<int32_t> st;
    McGeom m{};
    for (int l = 0; l < n_layers; ++l) {
        if (mc_geom(c, &convs[l], &m)) return HE_EINVAL;
        for (int32_t s : mc_conv_steps(convs[l], m)) st.push_back(s);
    }
    const int M = next_pow2_i(n_cls);
    for (int k = 1; k < M; ++k) st.push_back(k);                          // classifier
    for (int s = M; s < half; s <<= 1) st.push_back(s);
    std::vector<int32_t> uniq;
    for (int32_t s : st) {
        const int32_t v = ((s % half) + half) % half;
        if (v && std::find(uniq.begin(), uniq.end(), v) == uniq.end()) uniq.push_back(v);
    }
    uniq.push_back(HE_RELIN_KEY);
    for (int i = 0; i < (int)uniq.size() && i < cap && steps_out; ++i) steps_out[i] = uniq[i];
    return (int)uniq.size();
}

extern "C" int he_deep_batch(he_ctx* ctx, const he_ct* in, int B, const he_mc_conv* convs,
                             int n_layers, const int32_t* const* lowrank_w,
                             const int32_t* const* restore_w, const int32_t* fc_w, int n_cls,
                             he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!in || !convs || !lowrank_w || !restore_w || !fc_w || !out || B < 1 || n_layers < 1 ||
        n_cls < 1)
        return he_fail(ctx, HE_EINVAL, "he_deep: null or empty argument");
    int rc;
    std::vector<McGeom> gm(n_layers);
    for (int l = 0; l < n_layers; ++l) {
        if ((rc = mc_geom(ctx, &convs[l], &gm[l]))) return rc;
        if (l && (convs[l].C_in != convs[l - 1].O_c || convs[l].H != convs[0].H ||
                  convs[l].W != convs[0].W))
            return he_fail(ctx, HE_EINVAL, "he_deep: layer shapes do not chain");
    }
    const int L = ctx->L;
    for (int b = 0; b < B; ++b)
        if ((rc = check_ct(ctx, &out[b], L, -1, "he_deep output"))) return rc;
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    int widest = gm[0].n_in;
    for (auto& m : gm) widest = std::max(widest, m.n_out);
    // two ping-pong sets of activations in the context's network buffer
    const size_t set = (size_t)B * widest * ct;
    if ((rc = net_reserve(ctx, 2 * set))) return rc;
    uint64_t* bufs[2] = {(uint64_t*)ctx->net.base, (uint64_t*)ctx->net.base + set};
    auto cts_at = [&](uint64_t* p, int n) {
        std::vector<he_ct> v(n);
        for (int i = 0; i < n; ++i) v[i] = he_ct{p + (size_t)i * ct, 2u, (uint32_t)L, HE_NTT};
        return v;
    };
    std::vector<he_ct> cur(in, in + (size_t)B * gm[0].n_in);
    for (int l = 0; l < n_layers; ++l) {
        std::vector<he_ct> y = cts_at(bufs[0], B * gm[l].n_out);
        std::vector<he_ct> a = cts_at(bufs[1], B * gm[l].n_out);
        if ((rc = he_mc_conv_batch(ctx, cur.data(), B, lowrank_w[l], restore_w[l], &convs[l], y.data())))
            return rc;
        if ((rc = he_multiply_batch(ctx, y.data(), y.data(), (int)y.size(), a.data()))) return rc;
        cur = a;
    }
    // global sum pooling and the classifier as one linear map: logit_j = sum over (c, pixel) of
    // F[j][c] a[c, pixel], a fully connected layer over every activation of the last layer
    const McGeom& m = gm.back();
    const int C = convs[n_layers - 1].O_c, hw = convs[0].H * convs[0].W;
    std::vector<int32_t> ct_of((size_t)C * hw), pos((size_t)C * hw), Fx((size_t)n_cls * C * hw);
    for (int c = 0; c < C; ++c)
        for (int p = 0; p < hw; ++p) {
            const size_t i = (size_t)c * hw + p;
            ct_of[i] = c / m.g;
            pos[i] = (c % m.g) * m.Bk + p;
            for (int j = 0; j < n_cls; ++j) Fx[(size_t)j * C * hw + i] = fc_w[(size_t)j * C + c];
        }
    return he_fc_mc_batch(ctx, cur.data(), B, m.n_out, Fx.data(), ct_of.data(), pos.data(),
                          C * hw, n_cls, (int)(ctx->N / 2), out);
}
