// layer.cu -- the encrypted FFConv layer, FFConv packing DP-HI2C-CP (Sec. 4.2, Fig. 4).
//
// W1 (d x d, r = O'_c low-rank filters) under DensePack (Sec. 3.2, Fig. 1), the DP -> CP
// transition for a 1 x 1 kernel (Table III), W2 (1 x 1, r -> O_c) under ConvPack (Table II).
//
// HE_DP_DOT (the paper's DensePack dot products, Fig. 1a-c): for every low-rank channel c'
// and output position o the filter, zero-padded to the input size at its shifted location,
// multiplies the input; rotate-and-sum prod += rot(prod, 2^e), e < k, accumulates it, where
// 2^k covers the occupied slots (k = log2(N/2) and a final row swap when the input fills both
// rows; Table VIII's 7000 = 500 x 14 and 120 = 10 x 12).  One-hot masks then gather the r*S
// dot products into r ciphertexts (no rotation: Table III, DP-HI2C-CP, d = 1).
//
// HE_DP_DP (Table IX's DensePack-DensePack baseline): W1 as HE_DP_DOT, then W2 under DensePack
// as well (dp_dp_tail): the channels combined into one dense vector, one dense vector-row
// product and rotate-and-sum per output (c, o), one-hot masks gathering the results.
//
// HE_DP_SHIFT (hoisted taps): one hoisted rotation of the input per filter tap
// delta = (i - pad) I_w + (j - pad) and a plaintext per (c', tap) holding W1[c', ci, i, j] at
// the output base slots; channels folded with rotations by B_c 2^e.
//
// HE_DP_SHIFT_EXT (hoisted taps, extended-basis sums): the same slots and plaintexts, but the
// key-switched rotations are not divided by P one by one.  For every coefficient, one kernel
// forms each tap's inner product with its Galois key (plus P times the rotated c0), multiplies
// it by the tap plaintext lifted to Q u P and sums over taps for every channel in registers;
// one ModDown per (image, channel) follows.  Per image this replaces d^2 - 1 ModDowns (2K
// inverse and 2L forward transforms each) with r of them.
#include <algorithm>
#include <cstring>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

namespace {

struct LayoutInfo {
    int O_h, O_w, S, hw, B_c, taps, fold;
    int sum_depth;        // DP_DOT rotate-and-sum steps within a row
    bool both_rows;       // DP_DOT input spills into row 1 (adds the row swap)
};

int ceil_log2(long long x) {
    int k = 0;
    while ((1ll << k) < x) ++k;
    return k;
}

// After k rotate-and-sum steps slot o holds sum_{m < 2^k} prod[o + m]; valid when every
// output's zero-padded filter lies inside [o, o + 2^k).
bool window_covers(const he_layout& y, const LayoutInfo& li, int k) {
    for (int oh = 0; oh < li.O_h; ++oh)
        for (int ow = 0; ow < li.O_w; ++ow) {
            int o = oh * li.O_w + ow;
            int hmin = 1 << 30, hmax = -1, wmin = 1 << 30, wmax = -1;
            for (int i = 0; i < y.d; ++i) {
                int h = y.stride * oh + i - y.pad;
                if (h >= 0 && h < y.I_h) hmin = std::min(hmin, h), hmax = std::max(hmax, h);
                int w = y.stride * ow + i - y.pad;
                if (w >= 0 && w < y.I_w) wmin = std::min(wmin, w), wmax = std::max(wmax, w);
            }
            if (hmax < 0 || wmax < 0) continue;
            long long lo = (long long)hmin * y.I_w + wmin;
            long long hi = (long long)(y.I_c - 1) * li.hw + (long long)hmax * y.I_w + wmax;
            if (lo < o || hi >= o + (1ll << k)) return false;
        }
    return true;
}

int layout_info(const he_ctx* c, const he_layout* y, LayoutInfo* li, std::string* why) {
    if (y->I_c < 1 || y->I_h < 1 || y->I_w < 1 || y->d < 1 || y->stride < 1 || y->pad < 0 ||
        y->r < 1 || y->O_c < 1 ||
        (y->pack != HE_DP_DOT && y->pack != HE_DP_SHIFT && y->pack != HE_DP_SHIFT_EXT &&
         y->pack != HE_CP_CP && y->pack != HE_DP_DP)) {
        *why = "layout fields out of range";
        return HE_EINVAL;
    }
    li->O_h = (y->I_h + 2 * y->pad - y->d) / y->stride + 1;
    li->O_w = (y->I_w + 2 * y->pad - y->d) / y->stride + 1;
    if (y->I_h + 2 * y->pad < y->d || y->I_w + 2 * y->pad < y->d || li->O_h < 1 || li->O_w < 1) {
        *why = "filter larger than the padded input";
        return HE_EINVAL;
    }
    li->S = li->O_h * li->O_w;
    li->hw = y->I_h * y->I_w;
    li->B_c = y->I_c == 1 ? li->hw : (1 << ceil_log2(li->hw));
    li->taps = y->d * y->d;
    li->fold = ceil_log2(y->I_c);
    const long long half = c->N / 2;
    li->sum_depth = 0;
    li->both_rows = false;
    if (y->pack == HE_CP_CP) {
        if (li->S > c->N) {
            *why = "CP_CP output positions must fit in N slots";
            return HE_EINVAL;
        }
    } else if (y->pack == HE_DP_DOT || y->pack == HE_DP_DP) {
        long long span = (long long)y->I_c * li->hw;
        if (span > c->N || li->S > half) {
            *why = "DP_DOT input must fit in N slots and its output in N/2";
            return HE_EINVAL;
        }
        if (y->pack == HE_DP_DP && ((long long)y->r * li->S > half || y->modswitch)) {
            *why = "DP_DP needs r S <= N/2 (one dense vector) and no modulus switch";
            return HE_EINVAL;
        }
        const int full = ceil_log2(half);
        if (span > half) {
            li->sum_depth = full;
            li->both_rows = true;
        } else {
            int k = ceil_log2(span);
            li->sum_depth = (k < full && window_covers(*y, *li, k)) ? k : full;
        }
    } else {
        if ((long long)li->B_c * (1ll << li->fold) > half) {
            *why = "DP_SHIFT channel blocks must fit in one row of N/2 slots";
            return HE_EINVAL;
        }
    }
    return HE_OK;
}

// DP_DP: W2's rotate-and-sum depth, the smallest k2 with 2^k2 > (r - 1) S.
int dp_dp_k2(const he_layout& y, const LayoutInfo& li) {
    int k = 0;
    while ((1ll << k) <= (long long)(y.r - 1) * li.S) ++k;
    return k;
}

std::vector<int32_t> layer_steps(const he_layout& y, const LayoutInfo& li) {
    std::vector<int32_t> st;
    if (y.pack == HE_CP_CP) return st;   // ConvPack throughout: no rotation
    if (y.pack == HE_DP_DOT || y.pack == HE_DP_DP) {
        for (int e = 0; e < li.sum_depth; ++e) st.push_back(1 << e);
        if (li.both_rows) st.push_back(HE_ROW_SWAP);
        if (y.pack == HE_DP_DP) {             // combine, then W2's rotate-and-sum
            auto add = [&](int32_t v) {
                if (std::find(st.begin(), st.end(), v) == st.end()) st.push_back(v);
            };
            for (int c = 1; c < y.r; ++c) add(-c * li.S);
            for (int e = 0; e < dp_dp_k2(y, li); ++e) add(1 << e);
        }
    } else {
        for (int i = 0; i < y.d; ++i)
            for (int j = 0; j < y.d; ++j) {
                int dl = (i - y.pad) * y.I_w + (j - y.pad);
                if (dl != 0) st.push_back(dl);
            }
        for (int e = 0; e < li.fold; ++e) st.push_back(li.B_c << e);
    }
    return st;
}

// ---- slot vectors of the schedules' plaintexts (zeroed beforehand)

// DP_SHIFT: plaintext (c', i, j) holds W1[c', ci, i, j] at slot ci*B_c + (s oh) I_w + s ow for
// every output position whose input pixel (s oh + i - pad, s ow + j - pad) is inside.
// Low-rank weights small enough to travel as a kernel parameter: the slot kernels then read
// them from parameter space, and the layer needs no upload before its first kernel (an upload
// there would wait behind any large host-to-device copy the caller has queued).
constexpr int kW1Inline = 1024;
struct W1Inline {
    int32_t w[kW1Inline];
};

__global__ void k_dp_shift_slots(const int32_t* __restrict__ w1_dev, const __grid_constant__ W1Inline w1i,
                                 int I_c, int I_h, int I_w, int d,
                                 int s, int pad, int r, int O_h, int O_w, int B_c, int logN,
                                 int64_t* __restrict__ out) {
    const int32_t* w1 = w1_dev ? w1_dev : w1i.w;
    const int N = 1 << logN;
    const int pt = blockIdx.x;  // (c' * d + i) * d + j
    const int j = pt % d, i = (pt / d) % d, cp = pt / (d * d);
    const int per = I_c * O_h * O_w;
    for (int idx = threadIdx.x + blockIdx.y * blockDim.x; idx < per; idx += blockDim.x * gridDim.y) {
        int ow = idx % O_w, oh = (idx / O_w) % O_h, ci = idx / (O_w * O_h);
        int h = s * oh + i - pad, w = s * ow + j - pad;
        if (h < 0 || h >= I_h || w < 0 || w >= I_w) continue;
        int slot = ci * B_c + (s * oh) * I_w + s * ow;
        out[(size_t)pt * N + slot] = w1[((cp * I_c + ci) * d + i) * d + j];
    }
    (void)r;
}

// DP_DOT: plaintext (c', o) (index c' S + o) is filter c' zero-padded at output o; plaintext
// r S + o is the one-hot mask of slot o.
__global__ void k_dp_dot_slots(const int32_t* __restrict__ w1_dev, const __grid_constant__ W1Inline w1i,
                               int I_c, int I_h, int I_w, int d,
                               int s, int pad, int r, int O_w, int S, int logN,
                               int64_t* __restrict__ out) {
    const int32_t* w1 = w1_dev ? w1_dev : w1i.w;
    const int N = 1 << logN;
    const int pt = blockIdx.x;
    if (pt >= r * S) {
        if (threadIdx.x == 0 && blockIdx.y == 0) out[(size_t)pt * N + (pt - r * S)] = 1;
        return;
    }
    const int cp = pt / S, o = pt % S;
    const int oh = o / O_w, ow = o % O_w;
    const int per = I_c * d * d;
    const int hw = I_h * I_w;
    for (int idx = threadIdx.x + blockIdx.y * blockDim.x; idx < per; idx += blockDim.x * gridDim.y) {
        int j = idx % d, i = (idx / d) % d, ci = idx / (d * d);
        int h = s * oh + i - pad, w = s * ow + j - pad;
        if (h < 0 || h >= I_h || w < 0 || w >= I_w) continue;
        out[(size_t)pt * N + ci * hw + h * I_w + w] = w1[((cp * I_c + ci) * d + i) * d + j];
    }
}

// DP_DP: plaintext c S + o (row (c, o) of W2 under DensePack) holds W2[c][c'] at slot
// c' S + o of the dense vector, c' < r (slots zeroed beforehand).
__global__ void k_dp_dp_rows(const int32_t* __restrict__ w2, int r, int S, int logN,
                             int64_t* __restrict__ out) {
    const int N = 1 << logN;
    const int row = blockIdx.x, c = row / S, o = row - c * S;
    for (int cp = threadIdx.x; cp < r; cp += blockDim.x)
        out[(size_t)row * N + (size_t)cp * S + o] = w2[c * r + cp];
}

// Channel fold (input channels in blocks of B_c slots): acc <- acc + rot(acc, B_c 2^e); the
// result ends in A (A and A2 are swapped as needed).
int fold_channels(he_ctx* ctx, uint64_t*& A, uint64_t*& A2, int items, const LayoutInfo& li,
                  const RotBufs& rb, int chunk) {
    const size_t ct = 2 * (size_t)ctx->L * ctx->N;
    for (int e = 0; e < li.fold; ++e) {
        std::vector<uint64_t*> o(items);
        for (int q = 0; q < items; ++q) o[q] = A2 + (size_t)q * ct;
        int rc = rotate_contig(ctx, A, items, galois_elt(ctx, li.B_c << e), A, o, rb, chunk);
        if (rc) return rc;
        std::swap(A, A2);
    }
    return HE_OK;
}

}  // namespace

extern "C" int he_ffconv_required_steps(const he_ctx* ctx, const he_layout* layout,
                                        int32_t* steps_out, int cap) {
    if (!ctx || !layout) return HE_EINVAL;
    LayoutInfo li;
    std::string why;
    if (layout_info(ctx, layout, &li, &why)) return HE_EINVAL;
    std::vector<int32_t> st = layer_steps(*layout, li);
    for (int i = 0; i < (int)st.size() && i < cap && steps_out; ++i) steps_out[i] = st[i];
    return (int)st.size();
}

// Integer weights w[o][i] (o < n_out, i < n_in) -> Montgomery residues wm[(o n_in + i) L + l].
static std::vector<uint64_t> weights_mont(const he_ctx* ctx, const int32_t* w, int n_out, int n_in) {
    const int L = ctx->L;
    std::vector<uint64_t> wm((size_t)n_out * n_in * L);
    for (int o = 0; o < n_out; ++o)
        for (int i = 0; i < n_in; ++i)
            for (int l = 0; l < L; ++l) {
                const uint64_t q = ctx->mods[l];
                const int64_t v = w[(size_t)o * n_in + i];
                const uint64_t wr = v >= 0 ? (uint64_t)v % q : (q - ((uint64_t)(-v) % q)) % q;
                wm[((size_t)o * n_in + i) * L + l] = h_to_mont(wr, q);
            }
    return wm;
}

// W2 under ConvPack (Table II): ct_out[b][c] = sum_c' W2[c][c'] ct_w1[b][c'] with scalar
// plaintexts, from the channel results A [B][r][2][L][N]; then the optional modulus switch.
// d_wm: O_c r L words of the caller's scratch for the weights.
static int restore_layer(he_ctx* ctx, const uint64_t* A, int B, const he_layout& y,
                         const int32_t* restore_w, he_ct* ct_out, uint64_t* Y, uint64_t* last,
                         uint64_t* sprd, uint64_t* d_wm) {
    const int L = ctx->L, r = y.r, O_c = y.O_c;
    const size_t ct = 2 * (size_t)L * ctx->N;
    const std::vector<uint64_t> wm = weights_mont(ctx, restore_w, O_c, r);
    d_wm = (uint64_t*)upload_args(ctx, wm.data(), wm.size() * 8, d_wm);
    if (!d_wm) return he_fail(ctx, HE_ECUDA, "he_ffconv_layer: W2 upload failed");
    int rc;
    std::vector<uint64_t*> dst(B * O_c);
    for (int o = 0; o < B * O_c; ++o) {
        dst[o] = y.modswitch ? Y + (size_t)o * ct : ct_out[o].data;
        ct_out[o].domain = HE_NTT;
    }
    auto dp = upload_out_ptrs(ctx, dst);
    if (!dp) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
    phase_begin(ctx, HE_PHASE_RESTORE);
    launch_convpack(ctx, A, B, r, O_c, d_wm, dp, L);
    ctx->ops[0] += (uint64_t)B * O_c * r;
    ctx->ops[1] += (uint64_t)B * O_c * (r - 1);
    rc = he_launch_check(ctx, "he_ffconv_layer");
    if (rc) return rc;
    if (y.modswitch) {
        std::vector<const uint64_t*> xs(B * O_c);
        std::vector<uint64_t*> os(B * O_c);
        for (int o = 0; o < B * O_c; ++o) {
            xs[o] = Y + (size_t)o * ct;
            os[o] = ct_out[o].data;
        }
        if ((rc = rescale_items(ctx, xs, os, L, last, sprd))) return rc;
    }
    phase_end(ctx);
    return HE_OK;
}

// Scratch (u64 words) of the DP_DP tail for B images.
static size_t dp_dp_scratch(const he_ctx* ctx, const he_layout& y, const LayoutInfo& li, int B) {
    const size_t N = ctx->N, ct = 2 * (size_t)ctx->L * N, rows = (size_t)y.O_c * li.S;
    return 2 * (size_t)B * ct + 2 * (size_t)B * rows * ct + rows * (2 * N + (size_t)ctx->L * N) + 256;
}

// DP-DP tail (Table IX's DensePack-DensePack baseline) after the DP_DOT W1: the r channel
// ciphertexts A[b][c'] (y1[c', o] at slot o) are combined into one dense vector
// Y[b] = sum_c' rot(A[b][c'], -c' S); W2 under DensePack: z[b][c][o] = Y[b] * row(c, o),
// rotate-and-sum over 2^k2 > (r - 1) S slots (slot o then holds y2[c, o]), and the one-hot
// masks of the DP_DOT plaintexts gather the O_c S dot products into ct_out.  Buffers come from
// the arena the caller reserved (dp_dp_scratch words).
static int dp_dp_tail(he_ctx* ctx, const uint64_t* A, int B, const he_layout& y,
                      const LayoutInfo& li, const int32_t* restore_w, he_ct* ct_out,
                      const uint64_t* mask_pts, const RotBufs& rb, int chunk) {
    const int L = ctx->L, r = y.r, O_c = y.O_c, S = li.S, k2 = dp_dp_k2(y, li);
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    const int n_rows = O_c * S, n2 = B * n_rows;
    uint64_t* Xc = arena_take(ctx, (size_t)B * ct);
    uint64_t* Y = arena_take(ctx, (size_t)B * ct);
    uint64_t* Z = arena_take(ctx, (size_t)n2 * ct);
    uint64_t* Z2 = arena_take(ctx, (size_t)n2 * ct);
    int64_t* slots = (int64_t*)arena_take(ctx, (size_t)n_rows * N);
    uint64_t* tmp = arena_take(ctx, (size_t)n_rows * N);
    uint64_t* rows = arena_take(ctx, (size_t)n_rows * L * N);
    if (!rows) return he_fail(ctx, HE_ENOMEM, "he_ffconv_layer: DP_DP scratch");
    int rc;
    // combine the channels into one dense vector per image
    phase_begin(ctx, HE_PHASE_ROTATE);
    for (int b = 0; b < B; ++b)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(Y + (size_t)b * ct, A + (size_t)b * r * ct, ct * 8,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    for (int c = 1; c < r; ++c) {
        std::vector<uint64_t*> o(B);
        for (int b = 0; b < B; ++b) {
            HE_CHECK_CUDA(ctx, cudaMemcpyAsync(Xc + (size_t)b * ct, A + ((size_t)b * r + c) * ct, ct * 8,
                                               cudaMemcpyDeviceToDevice, ctx->stream));
            o[b] = Y + (size_t)b * ct;
        }
        if ((rc = rotate_contig(ctx, Xc, B, galois_elt(ctx, -c * S), Y, o, rb, chunk))) return rc;
    }
    phase_end(ctx);
    // W2 rows under DensePack
    phase_begin(ctx, HE_PHASE_ENCODE);
    const int32_t* d_w2 = (const int32_t*)upload_small(ctx, restore_w, (size_t)O_c * r * 4);
    if (!d_w2) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: W2 too large for staging");
    HE_CHECK_CUDA(ctx, cudaMemsetAsync(slots, 0, (size_t)n_rows * N * 8, ctx->stream));
    ++ctx->launches;
    k_dp_dp_rows<<<n_rows, 32, 0, ctx->stream>>>(d_w2, r, S, ctx->logN, slots);
    encode_device(ctx, slots, n_rows, tmp, rows, 1, L);
    phase_end(ctx);
    // z[b][c][o] = Y[b] * row(c, o), in launches of at most 8192 products (pointer tables)
    phase_begin(ctx, HE_PHASE_RESTORE);
    for (int s0 = 0; s0 < n2; s0 += 8192) {
        const int n = std::min(8192, n2 - s0);
        std::vector<const uint64_t*> xs(n), ps(n);
        std::vector<uint64_t*> os(n);
        for (int i = 0; i < n; ++i) {
            const int q = s0 + i, b = q / n_rows, row = q - b * n_rows;
            xs[i] = Y + (size_t)b * ct;
            ps[i] = rows + (size_t)row * L * N;
            os[i] = Z + (size_t)q * ct;
        }
        auto xp = upload_ptrs(ctx, xs);
        auto pp = upload_ptrs(ctx, ps);
        auto op = upload_out_ptrs(ctx, os);
        if (!xp || !pp || !op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        launch_mac(ctx, xp, pp, 1, nullptr, op, n, L);
    }
    phase_end(ctx);
    // rotate-and-sum: z <- z + rot(z, 2^e)
    phase_begin(ctx, HE_PHASE_ROTATE);
    for (int e = 0; e < k2; ++e) {
        std::vector<uint64_t*> o(n2);
        for (int q = 0; q < n2; ++q) o[q] = Z2 + (size_t)q * ct;
        if ((rc = rotate_contig(ctx, Z, n2, galois_elt(ctx, 1 << e), Z, o, rb, chunk))) return rc;
        std::swap(Z, Z2);
    }
    phase_end(ctx);
    // gather: ct_out[b][c] = sum_o z[b][c][o] * mask_o
    phase_begin(ctx, HE_PHASE_RESTORE);
    const int tmax = max_mac_terms(ctx);
    for (int o0 = 0; o0 < S; o0 += tmax) {
        const int T = std::min(tmax, S - o0);
        std::vector<const uint64_t*> mx((size_t)B * O_c * T), mp((size_t)B * O_c * T), ai;
        std::vector<uint64_t*> ao((size_t)B * O_c);
        for (int q = 0; q < B * O_c; ++q) {
            for (int t = 0; t < T; ++t) {
                mx[(size_t)q * T + t] = Z + ((size_t)q * S + o0 + t) * ct;
                mp[(size_t)q * T + t] = mask_pts + (size_t)(o0 + t) * L * N;
            }
            ao[q] = ct_out[q].data;
            ai.push_back(o0 ? ct_out[q].data : nullptr);
        }
        auto a1 = upload_ptrs(ctx, mx);
        auto a2 = upload_ptrs(ctx, mp);
        auto a3 = o0 ? upload_ptrs(ctx, ai) : nullptr;
        auto a4 = upload_out_ptrs(ctx, ao);
        if (!a1 || !a2 || !a4 || (o0 && !a3)) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        launch_mac(ctx, a1, a2, T, a3, a4, B * O_c, L);
    }
    for (int q = 0; q < B * O_c; ++q) ct_out[q].domain = HE_NTT;
    phase_end(ctx);
    // (rotate_contig counted the rotations, key switches and the additions that follow them)
    ctx->ops[0] += (uint64_t)B * 2 * n_rows;
    ctx->ops[1] += (uint64_t)B * O_c * (S - 1);
    return he_launch_check(ctx, "he_ffconv_layer");
}

// CP-HI2C-CP (Sec. 4.2 'ConvPack for W1', Fig. 5): ct_in holds K = d^2 I_c Im2Col column
// ciphertexts per image (image b's column k at b K + k).  W1 under ConvPack:
// ct_w1[b][c'] = sum_k W1[c'][k] ct_in[b][k]; the 1 x 1 W2 needs no regrouping (Table III,
// CP-HI2C-CP with d = 1: zero rotations).
static int cp_cp_layer(he_ctx* ctx, const he_ct* ct_in, int B, const int32_t* lowrank_w,
                       const int32_t* restore_w, const he_layout& y, const LayoutInfo& li,
                       he_ct* ct_out) {
    const int L = ctx->L, Lout = y.modswitch ? L - 1 : L;
    const int K = li.taps * y.I_c, r = y.r, O_c = y.O_c;
    int rc;
    for (int i = 0; i < B * K; ++i)
        if ((rc = check_ct(ctx, &ct_in[i], L, HE_NTT, "he_ffconv_layer input column"))) return rc;
    for (int o = 0; o < B * O_c; ++o)
        if ((rc = check_ct(ctx, &ct_out[o], Lout, -1, "he_ffconv_layer output"))) return rc;
    if (K > max_mac_terms(ctx)) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: too many columns");
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    size_t need = (size_t)B * K * ct + (size_t)B * r * ct +
                  (y.modswitch ? (size_t)B * O_c * (ct + 2 * N + 2 * (L - 1) * N) : 0) +
                  (size_t)(r * K + O_c * r) * L + 1024;                        // weights
    if ((rc = arena_reserve(ctx, need))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, (size_t)B * K * ct);
    uint64_t* A = arena_take(ctx, (size_t)B * r * ct);
    uint64_t* Y = y.modswitch ? arena_take(ctx, (size_t)B * O_c * ct) : nullptr;
    uint64_t* last = y.modswitch ? arena_take(ctx, (size_t)B * O_c * 2 * N) : nullptr;
    uint64_t* sprd = y.modswitch ? arena_take(ctx, (size_t)B * O_c * 2 * (L - 1) * N) : nullptr;
    for (int i = 0; i < B * K; ++i)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + (size_t)i * ct, ct_in[i].data, ct * 8,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    uint64_t* d_wm = arena_take(ctx, (size_t)r * K * L);
    uint64_t* d_wm2 = arena_take(ctx, (size_t)O_c * r * L);
    const std::vector<uint64_t> wm = weights_mont(ctx, lowrank_w, r, K);
    if (!d_wm || !d_wm2) return he_fail(ctx, HE_ENOMEM, "he_ffconv_layer: scratch");
    d_wm = (uint64_t*)upload_args(ctx, wm.data(), wm.size() * 8, d_wm);
    if (!d_wm) return he_fail(ctx, HE_ECUDA, "he_ffconv_layer: W1 upload failed");
    std::vector<uint64_t*> ao(B * r);
    for (int q = 0; q < B * r; ++q) ao[q] = A + (size_t)q * ct;
    auto op = upload_out_ptrs(ctx, ao);
    if (!op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
    phase_begin(ctx, HE_PHASE_TAPS);
    launch_convpack(ctx, X, B, K, r, d_wm, op, L);
    phase_end(ctx);
    ctx->ops[0] += (uint64_t)B * r * K;
    ctx->ops[1] += (uint64_t)B * r * (K - 1);
    return restore_layer(ctx, A, B, y, restore_w, ct_out, Y, last, sprd, d_wm2);
}

// W1 plaintexts of a layout (n_pt of them, pt_rows limbs each) from the integer weights:
// slot vectors on the device, then encoded in Montgomery form (slots, tmp: n_pt N words).
static int encode_w1(he_ctx* ctx, const he_layout& y, const LayoutInfo& li,
                     const int32_t* lowrank_w, int64_t* slots, uint64_t* tmp, uint64_t* pts) {
    const size_t N = ctx->N;
    const bool dot = y.pack == HE_DP_DOT || y.pack == HE_DP_DP;
    const int r = y.r, LK = ctx->L + ctx->K;
    const int pt_rows = y.pack == HE_DP_SHIFT_EXT ? LK : ctx->L;
    const int n_pt = dot ? r * li.S + li.S : r * li.taps;
    const size_t w1n = (size_t)r * y.I_c * y.d * y.d;
    // up to kW1Inline weights travel inline with the launch; larger sets are uploaded
    W1Inline w1i;
    const int32_t* d_w1 = nullptr;
    if (w1n <= (size_t)kW1Inline) {
        memcpy(w1i.w, lowrank_w, w1n * 4);
    } else {
        d_w1 = (const int32_t*)upload_small(ctx, lowrank_w, w1n * 4);
        if (!d_w1) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: W1 too large for staging");
    }
    HE_CHECK_CUDA(ctx, cudaMemsetAsync(slots, 0, (size_t)n_pt * N * 8, ctx->stream));
    ++ctx->launches;
    if (dot)
        k_dp_dot_slots<<<dim3(n_pt, 1), 256, 0, ctx->stream>>>(d_w1, w1i, y.I_c, y.I_h, y.I_w, y.d, y.stride,
                                                               y.pad, r, li.O_w, li.S, ctx->logN, slots);
    else
        k_dp_shift_slots<<<dim3(n_pt, 4), 256, 0, ctx->stream>>>(d_w1, w1i, y.I_c, y.I_h, y.I_w, y.d,
                                                                 y.stride, y.pad, r, li.O_h, li.O_w,
                                                                 li.B_c, ctx->logN, slots);
    encode_device(ctx, slots, n_pt, tmp, pts, 1, pt_rows);
    return HE_OK;
}

// The layer on B images; pre_pts, when given, holds the W1 plaintexts already encoded (a
// plan's), and the encode step is skipped.
static int layer_impl(he_ctx* ctx, const he_ct* ct_in, int B, const int32_t* lowrank_w,
                      const int32_t* restore_w, const he_layout* layout, he_ct* ct_out,
                      const uint64_t* pre_pts) {
    if (!ctx) return HE_EINVAL;
    if (!ct_in || !lowrank_w || !restore_w || !layout || !ct_out || B < 1)
        return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: null argument");
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: t is not 1 mod 2N");
    LayoutInfo li;
    std::string why;
    int rc = layout_info(ctx, layout, &li, &why);
    if (rc) return he_fail(ctx, rc, "he_ffconv_layer: " + why);
    const he_layout& y = *layout;
    const int L = ctx->L, Lout = y.modswitch ? L - 1 : L;
    if (y.modswitch && L < 2) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: modswitch needs two primes");
    if (y.pack == HE_CP_CP) return cp_cp_layer(ctx, ct_in, B, lowrank_w, restore_w, y, li, ct_out);
    for (int b = 0; b < B; ++b)
        if ((rc = check_ct(ctx, &ct_in[b], L, HE_NTT, "he_ffconv_layer input"))) return rc;
    for (int o = 0; o < B * y.O_c; ++o)
        if ((rc = check_ct(ctx, &ct_out[o], Lout, -1, "he_ffconv_layer output"))) return rc;
    const std::vector<int32_t> steps = layer_steps(y, li);
    std::vector<uint32_t> gs;
    for (int32_t st : steps) {
        uint32_t g = galois_elt(ctx, st);
        const uint64_t* k = nullptr;
        if ((rc = he_get_key(ctx, g, &k))) return rc;
        gs.push_back(g);
    }

    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    const int r = y.r, O_c = y.O_c;
    const bool dot = y.pack == HE_DP_DOT || y.pack == HE_DP_DP;   // DP_DP: W1 as DP_DOT
    const bool ext = y.pack == HE_DP_SHIFT_EXT;
    if (ext && li.taps > HE_MAX_TAPS) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer: too many filter taps");
    const int LK = L + ctx->K;
    const int pt_rows = ext ? LK : L;                          // extended plaintexts live in Q u P
    const int n_pt = dot ? r * li.S + li.S : r * li.taps;
    const int n_prod = dot ? B * r * li.S : (ext ? 0 : B * li.taps);   // ciphertexts fed to the MAC
    // ciphertexts key-switched per launch: all of them when the scratch allows (the
    // extended-basis schedule keeps every image's ModUp digits and channel sums at once)
    const int chunk = ext ? std::max(B * r, B)
                          : std::min(dot ? n_prod : (li.fold ? B * r : B), rotation_chunk(ctx));
    const int rot_items = chunk;
    const size_t ext_acc = ext ? (size_t)B * r * 2 * LK * N + (size_t)B * ct : 0;  // sums, P x
    // slots, tmp and plaintexts of the encode step (none when a plan holds the plaintexts)
    const size_t enc_words = pre_pts ? 0 : (size_t)n_pt * (2 * N + (size_t)pt_rows * N);
    size_t need = (size_t)B * ct                              // X
                  + enc_words
                  + (size_t)n_prod * ct * (dot ? 2 : 1)        // products (double buffer for DP_DOT)
                  + (size_t)2 * B * r * ct + ext_acc           // accumulators (double buffer)
                  + (size_t)rot_items * rot_scratch_per_item(ctx)
                  + (y.modswitch ? (size_t)B * O_c * (ct + 2 * N + 2 * (L - 1) * N) : 0)
                  + (y.pack == HE_DP_DP ? dp_dp_scratch(ctx, y, li, B) : 0)
                  + (size_t)O_c * r * L + 1024;                                 // W2 weights
    if ((rc = arena_reserve(ctx, need))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, (size_t)B * ct);
    int64_t* slots = pre_pts ? nullptr : (int64_t*)arena_take(ctx, (size_t)n_pt * N);
    uint64_t* tmp = pre_pts ? nullptr : arena_take(ctx, (size_t)n_pt * N);
    uint64_t* pts = pre_pts ? const_cast<uint64_t*>(pre_pts) : arena_take(ctx, (size_t)n_pt * pt_rows * N);
    uint64_t* PR = n_prod ? arena_take(ctx, (size_t)n_prod * ct) : nullptr;
    uint64_t* AX = ext ? arena_take(ctx, (size_t)B * r * 2 * LK * N) : nullptr;
    uint64_t* XP = ext ? arena_take(ctx, (size_t)B * ct) : nullptr;
    uint64_t* PR2 = dot ? arena_take(ctx, (size_t)n_prod * ct) : nullptr;
    uint64_t* A = arena_take(ctx, (size_t)B * r * ct);
    uint64_t* A2 = arena_take(ctx, (size_t)B * r * ct);
    RotBufs rb = rot_bufs_take(ctx, rot_items);
    uint64_t* Y = y.modswitch ? arena_take(ctx, (size_t)B * O_c * ct) : nullptr;
    uint64_t* last = y.modswitch ? arena_take(ctx, (size_t)B * O_c * 2 * N) : nullptr;
    uint64_t* sprd = y.modswitch ? arena_take(ctx, (size_t)B * O_c * 2 * (L - 1) * N) : nullptr;
    uint64_t* d_wm2 = arena_take(ctx, (size_t)O_c * r * L);
    if (!rb.v || !d_wm2 || (y.modswitch && !sprd))
        return he_fail(ctx, HE_ENOMEM, "he_ffconv_layer: scratch");

    // inputs -> contiguous X
    for (int b = 0; b < B; ++b)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + b * ct, ct_in[b].data, ct * 8, cudaMemcpyDeviceToDevice,
                                           ctx->stream));
    // (a1) plaintexts: slot vectors from the integer weights, encoded in Montgomery form
    if (!pre_pts) {
        phase_begin(ctx, HE_PHASE_ENCODE);
        if ((rc = encode_w1(ctx, y, li, lowrank_w, slots, tmp, pts))) return rc;
        phase_end(ctx);
    }

    if (dot) {
        // prod[b][c'][o] = X[b] * filter(c', o)
        std::vector<const uint64_t*> xs(n_prod), ps(n_prod);
        std::vector<uint64_t*> os(n_prod);
        for (int b = 0; b < B; ++b)
            for (int q = 0; q < r * li.S; ++q) {
                int it = b * r * li.S + q;
                xs[it] = X + b * ct;
                ps[it] = pts + (size_t)q * L * N;
                os[it] = PR + (size_t)it * ct;
            }
        auto xp = upload_ptrs(ctx, xs);
        auto pp = upload_ptrs(ctx, ps);
        auto op = upload_out_ptrs(ctx, os);
        if (!xp || !pp || !op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        phase_begin(ctx, HE_PHASE_TAPS);
        launch_mac(ctx, xp, pp, 1, nullptr, op, n_prod, L);
        phase_end(ctx);
        ctx->ops[0] += n_prod;
        // rotate-and-sum: PR2 = PR + rot(PR, step), then swap (the first sum_depth (+ row
        // swap) steps; DP_DP's list continues with its combine and W2 steps)
        phase_begin(ctx, HE_PHASE_ROTATE);
        const size_t n_w1_steps = (size_t)li.sum_depth + (li.both_rows ? 1 : 0);
        for (size_t si = 0; si < n_w1_steps; ++si) {
            std::vector<uint64_t*> outs(n_prod);
            for (int it = 0; it < n_prod; ++it) outs[it] = PR2 + (size_t)it * ct;
            if ((rc = rotate_contig(ctx, PR, n_prod, gs[si], PR, outs, rb, chunk))) return rc;
            std::swap(PR, PR2);
        }
        phase_end(ctx);
        // DP -> CP: ct_w1[b][c'] = sum_o prod[b][c'][o] * mask_o
        phase_begin(ctx, HE_PHASE_TAPS);
        const int tmax = max_mac_terms(ctx);
        for (int o0 = 0; o0 < li.S; o0 += tmax) {
            int T = std::min(tmax, li.S - o0);
            std::vector<const uint64_t*> mx((size_t)B * r * T), mp((size_t)B * r * T), ai;
            std::vector<uint64_t*> ao(B * r);
            for (int q = 0; q < B * r; ++q) {
                for (int t = 0; t < T; ++t) {
                    mx[(size_t)q * T + t] = PR + ((size_t)q * li.S + o0 + t) * ct;
                    mp[(size_t)q * T + t] = pts + (size_t)(r * li.S + o0 + t) * L * N;
                }
                ao[q] = A + (size_t)q * ct;
                ai.push_back(o0 ? A + (size_t)q * ct : nullptr);
            }
            auto a1 = upload_ptrs(ctx, mx);
            auto a2 = upload_ptrs(ctx, mp);
            auto a3 = o0 ? upload_ptrs(ctx, ai) : nullptr;
            auto a4 = upload_out_ptrs(ctx, ao);
            if (!a1 || !a2 || !a4 || (o0 && !a3)) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
            launch_mac(ctx, a1, a2, T, a3, a4, B * r, L);
        }
        phase_end(ctx);
        ctx->ops[0] += (uint64_t)B * r * li.S;
        ctx->ops[1] += (uint64_t)B * r * (li.S - 1);
    } else if (ext) {
        // one ModUp of every input's c1, then every tap's key switch and plaintext product
        // summed in Q u P, then one ModDown per (image, channel)
        phase_begin(ctx, HE_PHASE_MODUP);
        modup_items(ctx, X, B, 1u, rb);
        launch_scale_p(ctx, X, XP, B);
        phase_end(ctx);
        TapTable tt{};
        tt.n = li.taps;
        tt.r = r;
        tt.n_sub = 1;
        int tap = 0, nrot = 0;
        for (int i = 0; i < y.d; ++i)
            for (int j = 0; j < y.d; ++j, ++tap) {
                const int dl = (i - y.pad) * y.I_w + (j - y.pad);
                tt.key[tap] = nullptr;
                tt.g[tap] = 1u;
                if (dl == 0) continue;
                tt.g[tap] = galois_elt(ctx, dl);
                if ((rc = he_get_key(ctx, tt.g[tap], &tt.key[tap]))) return rc;
                ++nrot;
            }
        phase_begin(ctx, HE_PHASE_TAPS);
        launch_ks_mac_ext(ctx, rb.D, XP, pts, tt, AX, B);
        phase_end(ctx);
        const int items = B * r;
        phase_begin(ctx, HE_PHASE_MODDOWN);
        const size_t ext_ct = 2 * (size_t)LK * N;
        std::vector<uint64_t*> ao(items);
        for (int q = 0; q < items; ++q) ao[q] = A + (size_t)q * ct;
        auto op = upload_out_ptrs(ctx, ao);
        if (!op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        moddown_combine(ctx, AX, rb.v, items, nullptr, nullptr, op, 1u);
        phase_end(ctx);
        ctx->ops[0] += (uint64_t)B * r * li.taps;
        ctx->ops[1] += (uint64_t)B * r * (li.taps - 1);
        ctx->ops[2] += (uint64_t)B * nrot;
        ctx->ops[3] += (uint64_t)B * nrot;
        phase_begin(ctx, HE_PHASE_ROTATE);
        if ((rc = fold_channels(ctx, A, A2, B * r, li, rb, rot_items))) return rc;
        phase_end(ctx);
    } else {
        // hoisted rotations of every input by every non-zero tap offset
        std::vector<uint32_t> hg;
        std::vector<int> tap_of;
        std::vector<uint64_t*> outs;
        int tap = 0;
        for (int i = 0; i < y.d; ++i)
            for (int j = 0; j < y.d; ++j, ++tap) {
                int dl = (i - y.pad) * y.I_w + (j - y.pad);
                if (dl == 0) {
                    for (int b = 0; b < B; ++b)
                        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(PR + ((size_t)b * li.taps + tap) * ct, X + b * ct,
                                                           ct * 8, cudaMemcpyDeviceToDevice, ctx->stream));
                    continue;
                }
                hg.push_back(galois_elt(ctx, dl));
                for (int b = 0; b < B; ++b) outs.push_back(PR + ((size_t)b * li.taps + tap) * ct);
            }
        phase_begin(ctx, HE_PHASE_TAPS);
        for (int b0 = 0; b0 < B; b0 += rot_items) {
            int nb = std::min(rot_items, B - b0);
            std::vector<uint64_t*> o2;
            for (size_t s = 0; s < hg.size(); ++s)
                for (int b = 0; b < nb; ++b) o2.push_back(outs[s * B + b0 + b]);
            if ((rc = rotate_hoisted_contig(ctx, X + (size_t)b0 * ct, nb, hg, o2, rb))) return rc;
        }
        // acc[b][c'] = sum_tap R[b][tap] * pt[c'][tap]
        std::vector<const uint64_t*> mx((size_t)B * r * li.taps), mp((size_t)B * r * li.taps);
        std::vector<uint64_t*> ao(B * r);
        for (int b = 0; b < B; ++b)
            for (int cp = 0; cp < r; ++cp) {
                int q = b * r + cp;
                for (int t = 0; t < li.taps; ++t) {
                    mx[(size_t)q * li.taps + t] = PR + ((size_t)b * li.taps + t) * ct;
                    mp[(size_t)q * li.taps + t] = pts + ((size_t)cp * li.taps + t) * L * N;
                }
                ao[q] = A + (size_t)q * ct;
            }
        auto a1 = upload_ptrs(ctx, mx);
        auto a2 = upload_ptrs(ctx, mp);
        auto a4 = upload_out_ptrs(ctx, ao);
        if (!a1 || !a2 || !a4) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        launch_mac(ctx, a1, a2, li.taps, nullptr, a4, B * r, L);
        phase_end(ctx);
        ctx->ops[0] += (uint64_t)B * r * li.taps;
        ctx->ops[1] += (uint64_t)B * r * (li.taps - 1);
        phase_begin(ctx, HE_PHASE_ROTATE);
        if ((rc = fold_channels(ctx, A, A2, B * r, li, rb, rot_items))) return rc;
        phase_end(ctx);
    }

    if (y.pack == HE_DP_DP)
        return dp_dp_tail(ctx, A, B, y, li, restore_w, ct_out, pts + (size_t)r * li.S * L * N, rb,
                          rot_items);
    return restore_layer(ctx, A, B, y, restore_w, ct_out, Y, last, sprd, d_wm2);
}

extern "C" int he_ffconv_layer(he_ctx* ctx, const he_ct* ct_in, const int32_t* lowrank_w,
                               const int32_t* restore_w, const he_layout* layout, he_ct* ct_out) {
    return he_ffconv_layer_batch(ctx, ct_in, 1, lowrank_w, restore_w, layout, ct_out);
}

extern "C" int he_ffconv_layer_batch(he_ctx* ctx, const he_ct* ct_in, int B,
                                     const int32_t* lowrank_w, const int32_t* restore_w,
                                     const he_layout* layout, he_ct* ct_out) {
    return layer_impl(ctx, ct_in, B, lowrank_w, restore_w, layout, ct_out, nullptr);
}

// ------------------------------------------------------------------ layer plans

extern "C" int he_ffconv_plan(he_ctx* ctx, const int32_t* lowrank_w, const int32_t* restore_w,
                              const he_layout* layout, int32_t* plan_out) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_ffconv_plan");
    if (!lowrank_w || !restore_w || !layout || !plan_out)
        return he_fail(ctx, HE_EINVAL, "he_ffconv_plan: null argument");
    LayoutInfo li;
    std::string why;
    int rc = layout_info(ctx, layout, &li, &why);
    if (rc) return he_fail(ctx, rc, "he_ffconv_plan: " + why);
    const he_layout& y = *layout;
    he_ctx::LayerPlan pl;
    pl.layout = y;
    pl.w1.assign(lowrank_w, lowrank_w + (size_t)y.r * y.I_c * y.d * y.d);
    pl.w2.assign(restore_w, restore_w + (size_t)y.O_c * y.r);
    if (y.pack != HE_CP_CP) {
        const size_t N = ctx->N;
        const int pt_rows = y.pack == HE_DP_SHIFT_EXT ? ctx->L + ctx->K : ctx->L;
        const int n_pt = (y.pack == HE_DP_DOT || y.pack == HE_DP_DP) ? y.r * li.S + li.S : y.r * li.taps;
        if (cudaMalloc((void**)&pl.pts, (size_t)n_pt * pt_rows * N * 8) != cudaSuccess) {
            cudaGetLastError();
            return he_fail(ctx, HE_ENOMEM, "he_ffconv_plan: plaintext allocation failed");
        }
        if ((rc = arena_reserve(ctx, 2 * (size_t)n_pt * N + 64))) {
            cudaFree(pl.pts);
            return rc;
        }
        arena_reset(ctx);
        int64_t* slots = (int64_t*)arena_take(ctx, (size_t)n_pt * N);
        uint64_t* tmp = arena_take(ctx, (size_t)n_pt * N);
        if ((rc = encode_w1(ctx, y, li, pl.w1.data(), slots, tmp, pl.pts)) ||
            (rc = he_launch_check(ctx, "he_ffconv_plan"))) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(pl.pts);
            return rc;
        }
    }
    const int32_t id = ctx->next_plan++;
    ctx->plans[id] = std::move(pl);
    *plan_out = id;
    return HE_OK;
}

extern "C" int he_ffconv_layer_planned(he_ctx* ctx, int32_t plan, const he_ct* ct_in, int B,
                                       he_ct* ct_out) {
    if (!ctx) return HE_EINVAL;
    auto it = ctx->plans.find(plan);
    if (it == ctx->plans.end()) return he_fail(ctx, HE_EINVAL, "he_ffconv_layer_planned: no such plan");
    const he_ctx::LayerPlan& pl = it->second;
    if (ctx->rec) ctx->rec->g.plans.push_back(plan);     // a replay needs the plan alive
    return layer_impl(ctx, ct_in, B, pl.w1.data(), pl.w2.data(), &pl.layout, ct_out, pl.pts);
}

extern "C" int he_ffconv_plan_free(he_ctx* ctx, int32_t plan) {
    if (!ctx) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_ffconv_plan_free");
    auto it = ctx->plans.find(plan);
    if (it == ctx->plans.end()) return he_fail(ctx, HE_EINVAL, "he_ffconv_plan_free: no such plan");
    cudaStreamSynchronize(ctx->stream);
    if (it->second.pts) cudaFree(it->second.pts);
    ctx->plans.erase(it);
    return HE_OK;
}
