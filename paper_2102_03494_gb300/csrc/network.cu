// network.cu -- the three-layer encrypted network: FFConv layer, channel combine, x^2, fully
// connected, x^2, fully connected (the per-layer pipeline of Table VIII).
//
// Fully connected layer as DensePack dot products (Sec. 3: a fully connected layer is a
// convolution whose filter covers the whole input).  The input x_i sits at slot pos_i of row 0
// and repeats with period `per` (per = N/2 when it does not repeat).  With M the smallest
// power of two >= the output count m, the M diagonal plaintexts
//     diag_k[p] = F[p mod M][i]   where (p + k) mod per = pos_i and p mod M < m   (row 1: 0)
// give z = sum_{k<M} rot(x, k) * diag_k, in which slot p holds the terms of output p mod M
// whose input lies in the window p .. p + M - 1 (mod per).  Rotate-and-sum over the per/M
// windows of one period (z <- z + rot(z, M 2^e), e < log2(per/M)) leaves y_{p mod M} in every
// slot p (0 when p mod M >= m): the output repeats with period M, which is the input period
// of the next fully connected layer.  The M - 1 rotations of x share one ModUp and their
// plaintext products are summed in Q u P by the fused tap kernel (tapmac.cu), divided by P
// once; the rotate-and-sum steps are plain rotations of the whole batch per step.
//
// Channel combine: ct = ct_0 + sum_{c>=1} rot(ct_c, -c blk) puts channel c's values at
// c blk + slot(oh, ow) (Table VIII: "combine to one vector", O_c - 1 rotations).
#include <algorithm>
#include <string>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

namespace {

// slots[G M + k][p] = F[p mod M][inv[G][(p + k) mod per]] for p < N/2 with p mod M < m, else 0
// (G: input ciphertext, k: diagonal).
__global__ void k_fc_diag_slots(const int32_t* __restrict__ F, const int32_t* __restrict__ inv,
                                int m, int n_in, int M, int per, int logN,
                                int64_t* __restrict__ slots) {
    const int N = 1 << logN;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int G = blockIdx.y / M, k = blockIdx.y - G * M;
    int64_t v = 0;
    if (p < N / 2) {
        const int j = p & (M - 1);
        if (j < m) {
            const int i = inv[(size_t)G * per + ((p + k) & (per - 1))];
            if (i >= 0) v = F[(size_t)j * n_in + i];
        }
    }
    slots[(size_t)blockIdx.y * N + p] = v;
}

bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct ConvGeom {
    int O_h, O_w, S, blk;
    std::vector<int32_t> slot;   // output slot of (oh, ow) in the layer's own layout
};

// Output slots of the FFConv layer (row 0) and the combine block: the smallest power of two
// above every output slot.
ConvGeom conv_geom(const he_layout& y) {
    ConvGeom g;
    g.O_h = (y.I_h + 2 * y.pad - y.d) / y.stride + 1;
    g.O_w = (y.I_w + 2 * y.pad - y.d) / y.stride + 1;
    g.S = g.O_h * g.O_w;
    int top = 0;
    for (int oh = 0; oh < g.O_h; ++oh)
        for (int ow = 0; ow < g.O_w; ++ow) {
            const bool dense = y.pack == HE_DP_DOT || y.pack == HE_CP_CP || y.pack == HE_DP_DP;
            const int s = dense ? oh * g.O_w + ow : (y.stride * oh) * y.I_w + y.stride * ow;
            g.slot.push_back(s);
            top = std::max(top, s);
        }
    g.blk = next_pow2(top + 1);
    return g;
}

std::vector<int32_t> fc_steps(int m, int per) {
    const int M = next_pow2(m);
    std::vector<int32_t> st;
    for (int k = 1; k < M; ++k) st.push_back(k);
    for (int s = M; s < per; s <<= 1) st.push_back(s);
    return st;
}

int check_net(he_ctx* ctx, const he_net* net, ConvGeom* g) {
    if (!net) return he_fail(ctx, HE_EINVAL, "he_net: null shape");
    const int half = ctx->N / 2;
    if (net->conv.modswitch) return he_fail(ctx, HE_EINVAL, "he_net: the layer must keep every prime");
    if (net->conv.I_h < 1 || net->conv.I_w < 1 || net->conv.d < 1 || net->conv.stride < 1 ||
        net->conv.pad < 0 || net->conv.O_c < 1 || net->conv.I_h + 2 * net->conv.pad < net->conv.d ||
        net->conv.I_w + 2 * net->conv.pad < net->conv.d)
        return he_fail(ctx, HE_EINVAL, "he_net: layer shape out of range");
    *g = conv_geom(net->conv);
    if ((long long)net->conv.O_c * g->blk > half)
        return he_fail(ctx, HE_EINVAL, "he_net: the combined channels do not fit in one row");
    if (net->m1 < 1 || net->m2 < 1 || next_pow2(net->m1) > half ||
        next_pow2(net->m2) > next_pow2(net->m1))
        return he_fail(ctx, HE_EINVAL, "he_net: fully connected sizes do not fit their periods");
    return HE_OK;
}

}  // namespace

// Fully connected layer over n_ct input ciphertexts per image (the schedule in the file
// comment, taps of every input ciphertext summed in Q u P before the one ModDown): feature i
// sits at slot pos[i] of ciphertext ct_of[i], inside one period.
static int fc_core(he_ctx* ctx, const he_ct* in, int B, int n_ct, const int32_t* weights,
                   const int32_t* ct_of, const int32_t* pos, int n_feat, int n_out, int period,
                   he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!in || !weights || !pos || !out || B < 1 || n_ct < 1 || n_feat < 1 || n_out < 1)
        return he_fail(ctx, HE_EINVAL, "he_fc_layer: null or empty argument");
    if (!ctx->batching) return he_fail(ctx, HE_EINVAL, "he_fc_layer: t is not 1 mod 2N");
    const int half = ctx->N / 2, M = next_pow2(n_out);
    if (!is_pow2(period) || period > half || M > period)
        return he_fail(ctx, HE_EINVAL, "he_fc_layer: period must be a power of two, M <= period <= N/2");
    if (n_ct > 255) return he_fail(ctx, HE_EINVAL, "he_fc_layer: at most 255 input ciphertexts");
    std::vector<int32_t> inv((size_t)n_ct * period, -1);
    for (int i = 0; i < n_feat; ++i) {
        const int G = ct_of ? ct_of[i] : 0;
        if (G < 0 || G >= n_ct || pos[i] < 0 || pos[i] >= period || inv[(size_t)G * period + pos[i]] >= 0)
            return he_fail(ctx, HE_EINVAL, "he_fc_layer: positions must be distinct and inside one period");
        inv[(size_t)G * period + pos[i]] = i;
    }
    int rc;
    const int L = ctx->L, LK = L + ctx->K;
    for (int i = 0; i < B * n_ct; ++i)
        if ((rc = check_ct(ctx, &in[i], L, HE_NTT, "he_fc_layer input"))) return rc;
    for (int b = 0; b < B; ++b)
        if ((rc = check_ct(ctx, &out[b], L, -1, "he_fc_layer output"))) return rc;
    // keys: taps 1 .. M-1, then the sum steps
    const std::vector<int32_t> steps = fc_steps(n_out, period);
    std::vector<const uint64_t*> keys(steps.size());
    std::vector<uint32_t> gs(steps.size());
    for (size_t s = 0; s < steps.size(); ++s) {
        gs[s] = galois_elt(ctx, steps[s]);
        if ((rc = he_get_key(ctx, gs[s], &keys[s]))) return rc;
    }
    const size_t N = ctx->N, ct = 2 * (size_t)L * N, ext_ct = 2 * (size_t)LK * N;
    const int T = n_ct * M;                                  // taps: (input ciphertext, diagonal)
    const int n_chunks = (T + HE_MAX_TAPS - 1) / HE_MAX_TAPS;
    const size_t wn = (size_t)n_out * n_feat;
    const size_t items = (size_t)B * n_ct;
    const size_t need = items * ct * 2 + (size_t)B * ct * 2       // X, P x; A, A2
                        + (size_t)T * (2 * N + (size_t)LK * N)     // slots, tmp, plaintexts
                        + (size_t)B * ext_ct * (n_chunks > 1 ? 2 : 1)
                        + items * rot_scratch_per_item(ctx) + (wn + inv.size()) / 2 + 1 + 32 * 16;
    if ((rc = arena_reserve(ctx, need))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, items * ct);
    uint64_t* XP = arena_take(ctx, items * ct);
    uint64_t* A = arena_take(ctx, (size_t)B * ct);
    uint64_t* A2 = arena_take(ctx, (size_t)B * ct);
    int64_t* slots = (int64_t*)arena_take(ctx, (size_t)T * N);
    uint64_t* tmp = arena_take(ctx, (size_t)T * N);
    uint64_t* pts = arena_take(ctx, (size_t)T * LK * N);
    uint64_t* AX = arena_take(ctx, (size_t)B * ext_ct);
    uint64_t* AX2 = n_chunks > 1 ? arena_take(ctx, (size_t)B * ext_ct) : nullptr;
    int32_t* d_w = (int32_t*)arena_take(ctx, (wn + 1) / 2);
    int32_t* d_inv = (int32_t*)arena_take(ctx, (inv.size() + 1) / 2);
    RotBufs rb = rot_bufs_take(ctx, (int)items);
    if (!rb.v) return he_fail(ctx, HE_ENOMEM, "he_fc_layer: scratch");

    // diagonal plaintexts, lifted to Q u P in Montgomery form
    phase_begin(ctx, HE_PHASE_ENCODE);
    if ((rc = upload_host(ctx, d_w, weights, wn * 4))) return rc;
    if ((rc = upload_host(ctx, d_inv, inv.data(), inv.size() * 4))) return rc;
    ++ctx->launches;
    k_fc_diag_slots<<<dim3((unsigned)((N + 255) / 256), T), 256, 0, ctx->stream>>>(
        d_w, d_inv, n_out, n_feat, M, period, ctx->logN, slots);
    encode_device(ctx, slots, T, tmp, pts, 1, LK);
    phase_end(ctx);

    for (size_t i = 0; i < items; ++i)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + i * ct, in[i].data, ct * 8, cudaMemcpyDeviceToDevice,
                                           ctx->stream));
    phase_begin(ctx, HE_PHASE_MODUP);
    modup_items(ctx, X, (int)items, 1u, rb);
    launch_scale_p(ctx, X, XP, (int)items);
    phase_end(ctx);
    // sum over (G, k) of rot(x_G, k) diag_{G,k} in Q u P, at most HE_MAX_TAPS taps per launch
    phase_begin(ctx, HE_PHASE_TAPS);
    for (int c = 0; c < n_chunks; ++c) {
        const int t0 = c * HE_MAX_TAPS, nt = std::min(HE_MAX_TAPS, T - t0);
        TapTable tt{};
        tt.n = nt;
        tt.r = 1;
        tt.n_sub = n_ct;
        for (int u = 0; u < nt; ++u) {
            const int G = (t0 + u) / M, k = (t0 + u) - G * M;
            tt.key[u] = k ? keys[k - 1] : nullptr;
            tt.g[u] = k ? gs[k - 1] : 1u;
            tt.sub[u] = (uint8_t)G;
        }
        launch_ks_mac_ext(ctx, rb.D, XP, pts + (size_t)t0 * LK * N, tt, c ? AX2 : AX, B);
        if (c) {
            std::vector<const uint64_t*> xa(B), xb(B);
            std::vector<uint64_t*> xo(B);
            for (int b = 0; b < B; ++b) {
                xa[b] = AX + (size_t)b * ext_ct;
                xb[b] = AX2 + (size_t)b * ext_ct;
                xo[b] = AX + (size_t)b * ext_ct;
            }
            auto pa = upload_ptrs(ctx, xa);
            auto pb = upload_ptrs(ctx, xb);
            auto po = upload_out_ptrs(ctx, xo);
            if (!pa || !pb || !po) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
            launch_add_rows(ctx, pa, pb, po, B, LK);
        }
    }
    phase_end(ctx);
    // one ModDown per image
    phase_begin(ctx, HE_PHASE_MODDOWN);
    {
        std::vector<uint64_t*> ao(B);
        for (int b = 0; b < B; ++b) ao[b] = A + (size_t)b * ct;
        auto op = upload_out_ptrs(ctx, ao);
        if (!op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        moddown_combine(ctx, AX, rb.v, B, nullptr, nullptr, op, 1u);
    }
    phase_end(ctx);
    ctx->ops[0] += (uint64_t)B * T;
    ctx->ops[1] += (uint64_t)B * (T - 1);
    ctx->ops[2] += (uint64_t)B * n_ct * (M - 1);
    ctx->ops[3] += (uint64_t)B * n_ct * (M - 1);
    // rotate-and-sum over the windows of one period; the last step writes the outputs
    phase_begin(ctx, HE_PHASE_ROTATE);
    const int n_sum = (int)steps.size() - (M - 1);
    if (n_sum == 0) {
        for (int b = 0; b < B; ++b)
            HE_CHECK_CUDA(ctx, cudaMemcpyAsync(out[b].data, A + (size_t)b * ct, ct * 8,
                                               cudaMemcpyDeviceToDevice, ctx->stream));
    }
    for (int e = 0; e < n_sum; ++e) {
        std::vector<uint64_t*> o(B);
        for (int b = 0; b < B; ++b) o[b] = e == n_sum - 1 ? out[b].data : A2 + (size_t)b * ct;
        if ((rc = rotate_contig(ctx, A, B, gs[M - 1 + e], A, o, rb, B))) return rc;
        std::swap(A, A2);
    }
    phase_end(ctx);
    for (int b = 0; b < B; ++b) out[b].domain = HE_NTT;
    return he_launch_check(ctx, "he_fc_layer");
}

extern "C" int he_fc_layer_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* weights,
                                 const int32_t* pos, int n_in, int n_out, int period,
                                 he_ct* out) {
    return fc_core(ctx, in, B, 1, weights, nullptr, pos, n_in, n_out, period, out);
}

extern "C" int he_fc_mc_batch(he_ctx* ctx, const he_ct* in, int B, int n_ct,
                              const int32_t* weights, const int32_t* ct_of, const int32_t* pos,
                              int n_feat, int n_out, int period, he_ct* out) {
    if (ctx && !ct_of) return he_fail(ctx, HE_EINVAL, "he_fc_mc: null ciphertext indices");
    return fc_core(ctx, in, B, n_ct, weights, ct_of, pos, n_feat, n_out, period, out);
}

extern "C" int he_combine_batch(he_ctx* ctx, const he_ct* in, int B, int n_ch, int block,
                                he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!in || !out || B < 1 || n_ch < 1 || block < 0)
        return he_fail(ctx, HE_EINVAL, "he_combine: null or empty argument");
    int rc;
    const int L = ctx->L;
    for (int i = 0; i < B * n_ch; ++i)
        if ((rc = check_ct(ctx, &in[i], L, HE_NTT, "he_combine input"))) return rc;
    for (int b = 0; b < B; ++b)
        if ((rc = check_ct(ctx, &out[b], L, -1, "he_combine output"))) return rc;
    std::vector<uint32_t> gs(n_ch, 1u);
    const int half = ctx->N / 2;
    for (int c = 1; c < n_ch; ++c) {
        const long long st = (((long long)-c * block) % half + half) % half;
        gs[c] = galois_elt(ctx, (int32_t)st);
        const uint64_t* k = nullptr;
        if ((rc = he_get_key(ctx, gs[c], &k))) return rc;
    }
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    if ((rc = arena_reserve(ctx, (size_t)B * ct * 2 + (size_t)B * rot_scratch_per_item(ctx) + 32 * 8)))
        return rc;
    arena_reset(ctx);
    uint64_t* ACC = arena_take(ctx, (size_t)B * ct);
    uint64_t* X = arena_take(ctx, (size_t)B * ct);
    RotBufs rb = rot_bufs_take(ctx, B);
    if (!rb.v) return he_fail(ctx, HE_ENOMEM, "he_combine: scratch");
    for (int b = 0; b < B; ++b)
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(ACC + (size_t)b * ct, in[(size_t)b * n_ch].data, ct * 8,
                                           cudaMemcpyDeviceToDevice, ctx->stream));
    for (int c = 1; c < n_ch; ++c) {
        for (int b = 0; b < B; ++b)
            HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X + (size_t)b * ct, in[(size_t)b * n_ch + c].data,
                                               ct * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        std::vector<uint64_t*> o(B);
        for (int b = 0; b < B; ++b) o[b] = c == n_ch - 1 ? out[b].data : ACC + (size_t)b * ct;
        if ((rc = rotate_contig(ctx, X, B, gs[c], ACC, o, rb, B))) return rc;
    }
    if (n_ch == 1)
        for (int b = 0; b < B; ++b)
            HE_CHECK_CUDA(ctx, cudaMemcpyAsync(out[b].data, ACC + (size_t)b * ct, ct * 8,
                                               cudaMemcpyDeviceToDevice, ctx->stream));
    for (int b = 0; b < B; ++b) out[b].domain = HE_NTT;
    return he_launch_check(ctx, "he_combine");
}

extern "C" int he_net_required_steps(const he_ctx* ctx, const he_net* net, int32_t* steps_out,
                                     int cap) {
    if (!ctx || !net) return HE_EINVAL;
    he_ctx* c = const_cast<he_ctx*>(ctx);
    ConvGeom g;
    if (check_net(c, net, &g)) return HE_EINVAL;
    const int half = ctx->N / 2;
    int n = he_ffconv_required_steps(ctx, &net->conv, nullptr, 0);
    if (n < 0) return HE_EINVAL;
    std::vector<int32_t> st(n);
    if (n) he_ffconv_required_steps(ctx, &net->conv, st.data(), n);
    for (int ch = 1; ch < net->conv.O_c; ++ch)
        st.push_back((int32_t)(((-(long long)ch * g.blk) % half + half) % half));
    for (int32_t s : fc_steps(net->m1, half)) st.push_back(s);
    for (int32_t s : fc_steps(net->m2, next_pow2(net->m1))) st.push_back(s);
    std::vector<int32_t> uniq;
    for (int32_t s : st)
        if (std::find(uniq.begin(), uniq.end(), s) == uniq.end()) uniq.push_back(s);
    uniq.push_back(HE_RELIN_KEY);
    for (int i = 0; i < (int)uniq.size() && i < cap && steps_out; ++i) steps_out[i] = uniq[i];
    return (int)uniq.size();
}

extern "C" int he_net_batch(he_ctx* ctx, const he_ct* in, int B, const int32_t* lowrank_w,
                            const int32_t* restore_w, const int32_t* fc1_w, const int32_t* fc2_w,
                            const he_net* net, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    if (!in || !lowrank_w || !restore_w || !fc1_w || !fc2_w || !out || B < 1)
        return he_fail(ctx, HE_EINVAL, "he_net: null or empty argument");
    ConvGeom g;
    int rc = check_net(ctx, net, &g);
    if (rc) return rc;
    const int L = ctx->L, O_c = net->conv.O_c, half = ctx->N / 2;
    for (int b = 0; b < B; ++b)
        if ((rc = check_ct(ctx, &out[b], L, -1, "he_net output"))) return rc;
    const size_t N = ctx->N, ct = 2 * (size_t)L * N;
    // intermediates: layer outputs [B][O_c], then two ping-pong sets of B ciphertexts
    if ((rc = net_reserve(ctx, (size_t)B * ct * (O_c + 2)))) return rc;
    uint64_t* base = (uint64_t*)ctx->net.base;
    auto cts_at = [&](uint64_t* p, int n) {
        std::vector<he_ct> v(n);
        for (int i = 0; i < n; ++i) v[i] = he_ct{p + (size_t)i * ct, 2u, (uint32_t)L, HE_NTT};
        return v;
    };
    std::vector<he_ct> y = cts_at(base, B * O_c);
    std::vector<he_ct> u = cts_at(base + (size_t)B * O_c * ct, B);
    std::vector<he_ct> v = cts_at(base + (size_t)B * (O_c + 1) * ct, B);
    if ((rc = he_ffconv_layer_batch(ctx, in, B, lowrank_w, restore_w, &net->conv, y.data()))) return rc;
    if ((rc = he_combine_batch(ctx, y.data(), B, O_c, g.blk, u.data()))) return rc;
    if ((rc = he_multiply_batch(ctx, u.data(), u.data(), B, v.data()))) return rc;
    std::vector<int32_t> pos1;
    for (int ch = 0; ch < O_c; ++ch)
        for (int o = 0; o < g.S; ++o) pos1.push_back(ch * g.blk + g.slot[o]);
    if ((rc = he_fc_layer_batch(ctx, v.data(), B, fc1_w, pos1.data(), (int)pos1.size(), net->m1,
                                half, u.data())))
        return rc;
    if ((rc = he_multiply_batch(ctx, u.data(), u.data(), B, v.data()))) return rc;
    std::vector<int32_t> pos2(net->m1);
    for (int i = 0; i < net->m1; ++i) pos2[i] = i;
    return he_fc_layer_batch(ctx, v.data(), B, fc2_w, pos2.data(), net->m1, net->m2,
                             next_pow2(net->m1), out);
}
