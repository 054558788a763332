// eval.cu -- server-side evaluation: Galois key import/export, rotations (plain, batched,
// hoisted), MulPC/AddCC and modulus switching.
//
// Rotation by Galois element g (Sec. 3.2, Fig. 1b, as hybrid key switching):
//   plain:   T = INTT(perm_g(c1)); D_j = ModUp_j(T) (own digit rows: perm_g(c1));
//            u = sum_j D_j * key_j;  v = FastBConv_{P->Q}(INTT(u_P));
//            out = ((u_Q - NTT(v)) P^-1 + perm_g(c0), (u_Q - NTT(v)) P^-1)
//   hoisted: D_j = ModUp_j(INTT(c1)) once; per step u = sum_j perm_g(D_j) * key_j, same tail.
#include <algorithm>
#include <unordered_set>
#include <vector>

#include "eval.cuh"
#include "kernels.cuh"

// ------------------------------------------------------------------ keys

int he_get_key(he_ctx* ctx, uint32_t g, const uint64_t** key) {
    auto it = ctx->keys.find(g);
    if (it == ctx->keys.end())
        return he_fail(ctx, HE_ENOKEY, "no Galois key for element " + std::to_string(g));
    *key = it->second.dev;
    return HE_OK;
}

static int key_alloc(he_ctx* ctx, uint32_t g, uint64_t** dev) {
    auto it = ctx->keys.find(g);
    if (it != ctx->keys.end()) {
        *dev = it->second.dev;
        return HE_OK;
    }
    size_t bytes = (size_t)ctx->dnum * 2 * (ctx->L + ctx->K) * ctx->N * 8;
    uint64_t* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return he_fail(ctx, HE_ENOMEM, "key allocation failed");
    }
    ctx->keys[g] = GaloisKey{p};
    *dev = p;
    return HE_OK;
}

int he_key_for_generation(he_ctx* ctx, uint32_t g, uint64_t** dev) { return key_alloc(ctx, g, dev); }

extern "C" int he_export_galois(he_ctx* ctx, int32_t step, uint64_t* blob_out) {
    if (!ctx || !blob_out) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_export_galois");
    const uint64_t* key = nullptr;
    int rc = he_get_key(ctx, galois_elt(ctx, step), &key);
    if (rc) return rc;
    const size_t LK = ctx->L + ctx->K, total = (size_t)ctx->dnum * 2 * LK * ctx->N;
    if ((rc = arena_reserve(ctx, total))) return rc;
    arena_reset(ctx);
    uint64_t* tmp = arena_take(ctx, total);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(tmp, key, total * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    launch_from_mont(ctx, tmp, 1, (int)(2 * ctx->dnum * LK), (int)LK, 0);
    ntt_inverse(ctx, tmp, 2 * ctx->dnum, LK * ctx->N, (int)LK, 0);
    if ((rc = he_launch_check(ctx, "he_export_galois"))) return rc;
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(blob_out, tmp, total * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HE_OK;
}

extern "C" int he_load_keys(he_ctx* ctx, const uint64_t* blob, const int32_t* steps, int n_steps) {
    if (!ctx || n_steps < 0 || (n_steps > 0 && (!blob || !steps))) return HE_EINVAL;
    HE_NOT_RECORDING(ctx, "he_load_keys");
    const size_t LK = ctx->L + ctx->K, per = (size_t)ctx->dnum * 2 * LK * ctx->N;
    int rc = arena_reserve(ctx, 64);
    if (rc) return rc;
    arena_reset(ctx);
    int* bad = (int*)arena_take(ctx, 1);          // set when a residue is not below its modulus
    HE_CHECK_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    std::vector<uint32_t> loaded;
    for (int s = 0; s < n_steps; ++s) {
        uint64_t* key = nullptr;
        const uint32_t g = galois_elt(ctx, steps[s]);
        if ((rc = key_alloc(ctx, g, &key))) return rc;
        loaded.push_back(g);
        HE_CHECK_CUDA(ctx, cudaMemcpyAsync(key, blob + (size_t)s * per, per * 8,
                                           cudaMemcpyHostToDevice, ctx->stream));
        launch_check_range(ctx, key, (int)(2 * ctx->dnum * LK), (int)LK, bad);
        ntt_forward(ctx, key, 2 * ctx->dnum, LK * ctx->N, (int)LK, 0);
        launch_to_mont(ctx, key, 1, (int)(2 * ctx->dnum * LK), (int)LK, 0);
    }
    rc = he_launch_check(ctx, "he_load_keys");
    int h_bad = 0;
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HE_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!rc && h_bad) {                           // corrupted material: none of these keys stay
        for (uint32_t g : loaded) {
            auto it = ctx->keys.find(g);
            if (it != ctx->keys.end()) {
                if (it->second.dev) cudaFree(it->second.dev);
                ctx->keys.erase(it);
                ++ctx->keys_epoch;
            }
        }
        return he_fail(ctx, HE_EINVAL, "he_load_keys: key residue not below its modulus");
    }
    return rc;
}

// ------------------------------------------------------------------ rotation cores

size_t rot_scratch_per_item(const he_ctx* c) {
    const size_t L = c->L, LK = c->L + c->K;
    return (L + c->dnum * LK + 2 * LK + 2 * L) * (size_t)c->N;
}

RotBufs rot_bufs_take(he_ctx* c, int items) {
    const size_t N = c->N, L = c->L, LK = c->L + c->K;
    RotBufs b;
    b.T = arena_take(c, items * L * N);
    b.D = arena_take(c, items * c->dnum * LK * N);
    b.u = arena_take(c, items * 2 * LK * N);
    b.v = arena_take(c, items * 2 * L * N);
    return b;
}

// D <- ModUp of c1 of `items` contiguous ciphertexts X [items][2][L][N] (NTT domain), after
// the automorphism g_own (1 = none).
void modup_items(he_ctx* c, const uint64_t* X, int items, uint32_t g_own, const RotBufs& b) {
    const size_t N = c->N, L = c->L, LK = c->L + c->K;
    const size_t dstride = c->dnum * LK * N;
    launch_automorph(c, X + L * N, 2 * L * N, b.T, L * N, items, (int)L, g_own);
    if (c->bconv_fused) {
        // T <- y_i = [c1_i (Q_j/q_i)^-1]_{q_i} in coefficient form (the factor rides on N^-1);
        // each digit's own rows are c1 itself at perm positions; every other row is the
        // conversion, read by the forward NTT's first pass
        ntt_inverse_scaled(c, b.T, items, L * N, (int)L, 0, c->d_modup_ninv);
        launch_automorph(c, X + L * N, 2 * L * N, b.D, dstride, items, (int)L, g_own, c->alpha,
                         (int)LK);
        for (int j = 0; j < c->dnum; ++j) {
            const int i0 = j * c->alpha, i1 = std::min(i0 + c->alpha, c->L);
            const BConvSrc bc{b.T + (size_t)i0 * N, L * N, c->d_modup_c + (size_t)j * c->alpha * LK,
                              (int)LK, i1 - i0};
            ntt_forward_bconv(c, b.D + (size_t)j * LK * N, items, dstride, i0, 0, bc);
            ntt_forward_bconv(c, b.D + ((size_t)j * LK + i1) * N, items, dstride, (int)LK - i1, i1, bc);
        }
        return;
    }
    ntt_inverse(c, b.T, items, L * N, (int)L, 0);
    launch_modup(c, b.T, L * N, X + L * N, 2 * L * N, g_own, b.D, dstride, items);
    for (int j = 0; j < c->dnum; ++j) {
        int i0 = j * c->alpha, i1 = std::min(i0 + c->alpha, c->L);
        ntt_forward(c, b.D + (size_t)j * LK * N, items, dstride, i0, 0);
        ntt_forward(c, b.D + ((size_t)j * LK + i1) * N, items, dstride, (int)LK - i1, i1);
    }
}

// v <- the ModDown base conversion of the P limbs of u, NTT domain: u [items][2][L+K][N]
// (NTT domain; its P limbs are left in coefficient form, scaled), v [items][2][L][N].
void moddown_items(he_ctx* c, uint64_t* u, uint64_t* v, int items) {
    const size_t N = c->N, L = c->L, LK = c->L + c->K;
    if (c->bconv_fused) {
        ntt_inverse_scaled(c, u + L * N, items * 2, LK * N, c->K, (int)L, c->d_md_ninv);
        const BConvSrc bc{u + L * N, LK * N, c->d_md_c, (int)L, c->K};
        ntt_forward_bconv(c, v, items * 2, L * N, (int)L, 0, bc);
        return;
    }
    ntt_inverse(c, u + L * N, items * 2, LK * N, c->K, (int)L);
    launch_moddown_conv(c, u, 2 * LK * N, v, 2 * L * N, items);
    ntt_forward(c, v, items * 2, L * N, (int)L, 0);
}

// The ModDown of u and the key switch's last step: out[it] = (u_Q - conv(u_P)) P^-1
// (+ c0[it] at perm_g, + base[it]); v [items][2][L][N] is scratch.
void moddown_combine(he_ctx* c, uint64_t* u, uint64_t* v, int items, const uint64_t* const* c0p,
                     const uint64_t* const* basep, uint64_t* const* outp, uint32_t g) {
    const size_t N = c->N, L = c->L, LK = c->L + c->K;
    if (c->bconv_fused) {
        ntt_inverse_scaled(c, u + L * N, items * 2, LK * N, c->K, (int)L, c->d_md_ninv);
        const BConvSrc bc{u + L * N, LK * N, c->d_md_c, (int)L, c->K};
        const CombineDst cd{u, LK * N, c0p, basep, outp, c->d_md_pinv, (int)L, g};
        ntt_forward_bconv_combine(c, v, items * 2, L * N, (int)L, bc, cd);
        return;
    }
    moddown_items(c, u, v, items);
    launch_ks_combine(c, u, 2 * LK * N, v, 2 * L * N, c0p, basep, outp, items, g);
}

// Key switch of the prepared digits (read through perm g_ks) and the rotation's tail:
// out[it] = (u - v) P^-1 + perm_g(c0[it]) (+ base[it]).
void ks_items(he_ctx* c, int items, const uint64_t* key, uint32_t g_ks, uint32_t g,
              const uint64_t* const* c0p, const uint64_t* const* basep, uint64_t* const* outp,
              const RotBufs& b) {
    const size_t N = c->N, L = c->L, LK = c->L + c->K;
    launch_ks_inner(c, b.D, c->dnum * LK * N, key, b.u, 2 * LK * N, items, g_ks);
    moddown_combine(c, b.u, b.v, items, c0p, basep, outp, g);
}

const uint64_t* const* upload_ptrs(he_ctx* c, const std::vector<const uint64_t*>& v) {
    return (const uint64_t* const*)upload_small(c, v.data(), v.size() * sizeof(void*));
}

uint64_t* const* upload_out_ptrs(he_ctx* c, const std::vector<uint64_t*>& v) {
    return (uint64_t* const*)upload_small(c, v.data(), v.size() * sizeof(void*));
}

// Plain rotation of `items` contiguous ciphertexts X by Galois element g, chunked so that the
// scratch stays bounded; out[it] (+= base[it] when base_contig) are contiguous or listed.
int rotate_contig(he_ctx* c, const uint64_t* X, int items, uint32_t g, const uint64_t* base,
                  const std::vector<uint64_t*>& outs, const RotBufs& b, int chunk) {
    const uint64_t* key = nullptr;
    int rc = he_get_key(c, g, &key);
    if (rc) return rc;
    const size_t ct = 2 * (size_t)c->L * c->N;
    for (int s = 0; s < items; s += chunk) {
        int n = std::min(chunk, items - s);
        std::vector<const uint64_t*> c0(n), bs(n);
        std::vector<uint64_t*> o(n);
        for (int i = 0; i < n; ++i) {
            c0[i] = X + (size_t)(s + i) * ct;
            bs[i] = base ? base + (size_t)(s + i) * ct : nullptr;
            o[i] = outs[s + i];
        }
        auto c0p = upload_ptrs(c, c0);
        auto bp = base ? upload_ptrs(c, bs) : nullptr;
        auto op = upload_out_ptrs(c, o);
        if (!c0p || !op || (base && !bp)) return he_fail(c, HE_ECUDA, "pointer table upload failed");
        modup_items(c, X + (size_t)s * ct, n, g, b);
        ks_items(c, n, key, 1u, g, c0p, bp, op, b);
    }
    c->ops[2] += items;
    c->ops[3] += items;
    if (base) c->ops[1] += items;
    return he_launch_check(c, "rotation");
}

int rotation_chunk(const he_ctx* c) {
    // keep the key-switching scratch of one chunk near 1 GiB
    size_t per = rot_scratch_per_item(c) * 8;
    size_t ch = ((size_t)1 << 30) / per;
    return (int)std::max<size_t>(1, std::min<size_t>(ch, 4096));
}

// ------------------------------------------------------------------ public rotations

static int gather_inputs(he_ctx* c, const he_ct* in, int n, uint64_t* X) {
    const size_t ct = 2 * (size_t)c->L * c->N;
    for (int i = 0; i < n; ++i)
        HE_CHECK_CUDA(c, cudaMemcpyAsync(X + i * ct, in[i].data, ct * 8, cudaMemcpyDeviceToDevice,
                                         c->stream));
    return HE_OK;
}

extern "C" int he_rotate_batch(he_ctx* ctx, const he_ct* in, int n, int32_t step, he_ct* out) {
    if (!ctx || !in || !out || n < 1) return ctx ? he_fail(ctx, HE_EINVAL, "he_rotate_batch: arguments") : HE_EINVAL;
    for (int i = 0; i < n; ++i) {
        int rc = check_ct(ctx, &in[i], ctx->L, HE_NTT, "he_rotate input");
        if (!rc) rc = check_ct(ctx, &out[i], ctx->L, -1, "he_rotate output");
        if (rc) return rc;
    }
    const uint32_t g = galois_elt(ctx, step);
    const uint64_t* key = nullptr;
    int rc = he_get_key(ctx, g, &key);
    if (rc) return rc;
    const int chunk = std::min(n, rotation_chunk(ctx));
    const size_t ct = 2 * (size_t)ctx->L * ctx->N;
    if ((rc = arena_reserve(ctx, n * ct + chunk * rot_scratch_per_item(ctx) + 64))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, n * ct);
    RotBufs b = rot_bufs_take(ctx, chunk);
    if ((rc = gather_inputs(ctx, in, n, X))) return rc;
    std::vector<uint64_t*> outs(n);
    for (int i = 0; i < n; ++i) {
        outs[i] = out[i].data;
        out[i].domain = HE_NTT;
    }
    return rotate_contig(ctx, X, n, g, nullptr, outs, b, chunk);
}

extern "C" int he_automorphism(he_ctx* ctx, const he_ct* in, int n, int32_t step, he_ct* out) {
    if (!ctx || !in || !out || n < 1)
        return ctx ? he_fail(ctx, HE_EINVAL, "he_automorphism: arguments") : HE_EINVAL;
    for (int i = 0; i < n; ++i) {
        int rc = check_ct(ctx, &in[i], 0, HE_NTT, "he_automorphism input");
        if (!rc) rc = check_ct(ctx, &out[i], (int)in[i].n_limbs, -1, "he_automorphism output");
        if (rc) return rc;
        if (in[i].data == out[i].data)
            return he_fail(ctx, HE_EINVAL, "he_automorphism: input and output must not alias");
    }
    const uint32_t g = galois_elt(ctx, step);
    const size_t N = ctx->N, lv = in[0].n_limbs, poly = lv * N;
    // ciphertexts stored back to back (inputs and outputs alike, one level): one launch over
    // all 2 n polynomials; otherwise one launch per ciphertext
    bool contig = true;
    for (int i = 0; i < n && contig; ++i)
        contig = in[i].n_limbs == lv && in[i].data == in[0].data + 2 * poly * i &&
                 out[i].data == out[0].data + 2 * poly * i;
    if (contig) {
        launch_automorph(ctx, in[0].data, poly, out[0].data, poly, 2 * n, (int)lv, g);
    } else {
        for (int i = 0; i < n; ++i) {
            const size_t p = (size_t)in[i].n_limbs * N;
            launch_automorph(ctx, in[i].data, p, out[i].data, p, 2, (int)in[i].n_limbs, g);
        }
    }
    for (int i = 0; i < n; ++i) out[i].domain = HE_NTT;
    return he_launch_check(ctx, "he_automorphism");
}

extern "C" int he_rotate(he_ctx* ctx, const he_ct* in, int32_t step, he_ct* out) {
    return he_rotate_batch(ctx, in, 1, step, out);
}

// Hoisted rotations of `items` contiguous ciphertexts by each of `steps`; out pointer
// outs[s * items + it].
int rotate_hoisted_contig(he_ctx* c, const uint64_t* X, int items, const std::vector<uint32_t>& gs,
                          const std::vector<uint64_t*>& outs, const RotBufs& b) {
    std::vector<const uint64_t*> keys(gs.size());
    for (size_t s = 0; s < gs.size(); ++s) {
        int rc = he_get_key(c, gs[s], &keys[s]);
        if (rc) return rc;
    }
    const size_t ct = 2 * (size_t)c->L * c->N;
    std::vector<const uint64_t*> c0(items);
    for (int i = 0; i < items; ++i) c0[i] = X + (size_t)i * ct;
    auto c0p = upload_ptrs(c, c0);
    if (!c0p) return he_fail(c, HE_ECUDA, "pointer table upload failed");
    modup_items(c, X, items, 1u, b);
    for (size_t s = 0; s < gs.size(); ++s) {
        std::vector<uint64_t*> o(outs.begin() + s * items, outs.begin() + (s + 1) * items);
        auto op = upload_out_ptrs(c, o);
        if (!op) return he_fail(c, HE_ECUDA, "pointer table upload failed");
        ks_items(c, items, keys[s], gs[s], gs[s], c0p, nullptr, op, b);
    }
    c->ops[2] += (uint64_t)items * gs.size();
    c->ops[3] += (uint64_t)items * gs.size();
    return he_launch_check(c, "hoisted rotation");
}

extern "C" int he_rotate_hoisted_batch(he_ctx* ctx, const he_ct* in, int n, const int32_t* steps,
                                       int h, he_ct* outs) {
    if (!ctx || !in || !steps || !outs || n < 1 || h < 1)
        return ctx ? he_fail(ctx, HE_EINVAL, "he_rotate_hoisted_batch: arguments") : HE_EINVAL;
    std::vector<uint32_t> gs(h);
    for (int s = 0; s < h; ++s) gs[s] = galois_elt(ctx, steps[s]);
    // inputs are gathered chunk by chunk, so an output written for one chunk must not be a
    // later chunk's input
    std::unordered_set<const uint64_t*> ins;
    for (int i = 0; i < n; ++i) ins.insert(in[i].data);
    for (size_t j = 0; j < (size_t)n * h; ++j)
        if (ins.count(outs[j].data))
            return he_fail(ctx, HE_EINVAL, "he_rotate_hoisted_batch: an output aliases an input");
    for (int i = 0; i < n; ++i) {
        int rc = check_ct(ctx, &in[i], ctx->L, HE_NTT, "he_rotate_hoisted_batch input");
        if (rc) return rc;
        for (int s = 0; s < h; ++s)
            if ((rc = check_ct(ctx, &outs[(size_t)i * h + s], ctx->L, -1, "he_rotate_hoisted_batch output")))
                return rc;
    }
    const size_t ct = 2 * (size_t)ctx->L * ctx->N;
    const int chunk = std::min(n, rotation_chunk(ctx));
    int rc = arena_reserve(ctx, chunk * ct + chunk * rot_scratch_per_item(ctx) + 64);
    if (rc) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, chunk * ct);
    RotBufs b = rot_bufs_take(ctx, chunk);
    for (int i0 = 0; i0 < n; i0 += chunk) {
        const int items = std::min(chunk, n - i0);
        if ((rc = gather_inputs(ctx, in + i0, items, X))) return rc;
        std::vector<uint64_t*> o((size_t)h * items);   // step-major, as rotate_hoisted_contig takes them
        for (int it = 0; it < items; ++it)
            for (int s = 0; s < h; ++s) {
                he_ct& oc = outs[(size_t)(i0 + it) * h + s];
                o[(size_t)s * items + it] = oc.data;
                oc.domain = HE_NTT;
            }
        if ((rc = rotate_hoisted_contig(ctx, X, items, gs, o, b))) return rc;
    }
    return HE_OK;
}

extern "C" int he_rotate_hoisted(he_ctx* ctx, const he_ct* in, const int32_t* steps, int h,
                                 he_ct* outs) {
    if (!ctx || !in || !steps || !outs || h < 1) return ctx ? he_fail(ctx, HE_EINVAL, "he_rotate_hoisted: arguments") : HE_EINVAL;
    int rc = check_ct(ctx, in, ctx->L, HE_NTT, "he_rotate_hoisted input");
    if (rc) return rc;
    std::vector<uint32_t> gs(h);
    std::vector<uint64_t*> o(h);
    for (int s = 0; s < h; ++s) {
        if ((rc = check_ct(ctx, &outs[s], ctx->L, -1, "he_rotate_hoisted output"))) return rc;
        gs[s] = galois_elt(ctx, steps[s]);
        o[s] = outs[s].data;
        outs[s].domain = HE_NTT;
    }
    const size_t ct = 2 * (size_t)ctx->L * ctx->N;
    if ((rc = arena_reserve(ctx, ct + rot_scratch_per_item(ctx) + 64))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, ct);
    RotBufs b = rot_bufs_take(ctx, 1);
    if ((rc = gather_inputs(ctx, in, 1, X))) return rc;
    return rotate_hoisted_contig(ctx, X, 1, gs, o, b);
}

// ------------------------------------------------------------------ MulPC / AddCC

int max_mac_terms(const he_ctx* c) {
    uint64_t qmax = 0;
    for (int i = 0; i < c->L; ++i) qmax = std::max(qmax, c->mods[i]);
    uint64_t t = (~0ull) / qmax;   // sum of t products of residues < q stays below q 2^64
    return (int)std::min<uint64_t>(t > 1 ? t - 1 : 1, 1u << 20);
}

extern "C" int he_mul_plain_acc(he_ctx* ctx, const he_ct* cts, const uint64_t* pts, int n,
                                he_ct* acc) {
    if (!ctx || !cts || !pts || !acc || n < 1) return ctx ? he_fail(ctx, HE_EINVAL, "he_mul_plain_acc: arguments") : HE_EINVAL;
    int rc = check_ct(ctx, acc, 0, HE_NTT, "he_mul_plain_acc acc");
    if (rc) return rc;
    const int Lv = acc->n_limbs;
    for (int i = 0; i < n; ++i)
        if ((rc = check_ct(ctx, &cts[i], Lv, HE_NTT, "he_mul_plain_acc ct"))) return rc;
    const size_t N = ctx->N, L = ctx->L;
    if ((rc = arena_reserve(ctx, (size_t)n * L * N + 64))) return rc;
    arena_reset(ctx);
    uint64_t* pm = arena_take(ctx, (size_t)n * L * N);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(pm, pts, (size_t)n * L * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    launch_to_mont(ctx, pm, n, (int)L, (int)L, 0);
    const int tmax = max_mac_terms(ctx);
    for (int s = 0; s < n; s += tmax) {
        int T = std::min(tmax, n - s);
        std::vector<const uint64_t*> X(T), P(T);
        for (int t = 0; t < T; ++t) {
            X[t] = cts[s + t].data;
            P[t] = pm + (size_t)(s + t) * L * N;
        }
        auto xp = upload_ptrs(ctx, X);
        auto pp = upload_ptrs(ctx, P);
        auto ap = upload_ptrs(ctx, {acc->data});
        auto op = upload_out_ptrs(ctx, {acc->data});
        if (!xp || !pp || !ap || !op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
        launch_mac(ctx, xp, pp, T, ap, op, 1, Lv);
    }
    ctx->ops[0] += n;
    ctx->ops[1] += n;
    return he_launch_check(ctx, "he_mul_plain_acc");
}

extern "C" int he_add(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    int rc = check_ct(ctx, a, 0, -1, "he_add a");
    if (!rc) rc = check_ct(ctx, b, a->n_limbs, a->domain, "he_add b");
    if (!rc) rc = check_ct(ctx, out, a->n_limbs, -1, "he_add out");
    if (rc) return rc;
    auto ap = upload_ptrs(ctx, {a->data});
    auto bp = upload_ptrs(ctx, {b->data});
    auto op = upload_out_ptrs(ctx, {out->data});
    if (!ap || !bp || !op) return he_fail(ctx, HE_ECUDA, "pointer table upload failed");
    launch_add(ctx, ap, bp, op, 1, a->n_limbs);
    out->domain = a->domain;
    ctx->ops[1] += 1;
    return he_launch_check(ctx, "he_add");
}

// ------------------------------------------------------------------ modulus switching

// out[it] (level Lv-1) = round(x[it] / q_{Lv-1}) for `items` ciphertexts at level Lv listed in
// xs (NTT domain); outs must not alias xs.
int rescale_items(he_ctx* c, const std::vector<const uint64_t*>& xs,
                  const std::vector<uint64_t*>& outs, int Lv, uint64_t* last, uint64_t* s) {
    const int items = (int)xs.size();
    const size_t N = c->N;
    auto xp = upload_ptrs(c, xs);
    auto op = upload_out_ptrs(c, outs);
    if (!xp || !op) return he_fail(c, HE_ECUDA, "pointer table upload failed");
    launch_gather_last(c, xp, last, items, Lv);
    ntt_inverse(c, last, items * 2, N, 1, Lv - 1);
    launch_rescale_spread(c, last, s, items, Lv);
    ntt_forward(c, s, items * 2, (size_t)(Lv - 1) * N, Lv - 1, 0);
    launch_rescale_combine(c, xp, s, op, items, Lv);
    return he_launch_check(c, "rescale");
}

extern "C" int he_rescale(he_ctx* ctx, const he_ct* in, he_ct* out) {
    if (!ctx) return HE_EINVAL;
    int rc = check_ct(ctx, in, 0, HE_NTT, "he_rescale input");
    if (rc) return rc;
    const int Lv = in->n_limbs;
    if (Lv < 2) return he_fail(ctx, HE_EINVAL, "he_rescale: needs at least two limbs");
    if ((rc = check_ct(ctx, out, Lv - 1, -1, "he_rescale output"))) return rc;
    const size_t N = ctx->N;
    if ((rc = arena_reserve(ctx, 2 * Lv * N + 2 * N + 2 * (Lv - 1) * N + 64))) return rc;
    arena_reset(ctx);
    uint64_t* X = arena_take(ctx, 2 * Lv * N);
    uint64_t* last = arena_take(ctx, 2 * N);
    uint64_t* s = arena_take(ctx, 2 * (Lv - 1) * N);
    HE_CHECK_CUDA(ctx, cudaMemcpyAsync(X, in->data, 2 * Lv * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    out->domain = HE_NTT;
    return rescale_items(ctx, {X}, {out->data}, Lv, last, s);
}
