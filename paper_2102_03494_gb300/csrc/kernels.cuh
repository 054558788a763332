// kernels.cuh -- launchers of the element-wise / base-conversion kernels (kernels.cu).
#pragma once

#include "he_internal.cuh"

#define HE_DEC_MAX_WORDS 31
#define HE_MAX_TAPS 64

// Per-tap rotation data of the extended-basis tap MAC (passed by value as a kernel argument):
// the key (null for the zero offset) and Galois element of each tap, tap count, channels, and
// for inputs of several ciphertexts per image the one each tap reads: tap t of image b uses
// the ModUp digits and P x of item b n_sub + sub[t] (n_sub = 1, sub = 0 for one ciphertext).
struct TapTable {
    const uint64_t* key[HE_MAX_TAPS];
    uint32_t g[HE_MAX_TAPS];
    uint8_t sub[HE_MAX_TAPS];
    int n;
    int r;
    int n_sub;
};

// XP ([B][2][L][N]) <- P times the inputs X, per ciphertext limb.  B counts ciphertexts.
void launch_scale_p(he_ctx* c, const uint64_t* X, uint64_t* XP, int B);
// Extended-basis tap MAC over B images (dnum <= 8); XP from launch_scale_p.  Uses the
// bulk-copy pipelined kernel (tapmac.cu) when N >= 256, else the register-only kernel.
void launch_ks_mac_ext(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                       const TapTable& tt, uint64_t* A, int B);
bool tapmac_bulk_supported(const he_ctx* c);
void launch_ks_mac_ext_bulk(he_ctx* c, const uint64_t* D, const uint64_t* XP, const uint64_t* pts,
                            const TapTable& tt, uint64_t* A, int B);

// out row r = in row r at perm_g positions; with alpha > 0, out row (r / alpha) lk + r.
void launch_automorph(he_ctx* c, const uint64_t* in, size_t in_stride, uint64_t* out,
                      size_t out_stride, int items, int rows, uint32_t g, int alpha = 0,
                      int lk = 0);
void launch_modup(he_ctx* c, const uint64_t* x_coeff, size_t xc_stride, const uint64_t* x_ntt,
                  size_t xn_stride, uint32_t g_own, uint64_t* out, size_t out_stride, int items);
void launch_ks_inner(he_ctx* c, const uint64_t* D, size_t d_stride, const uint64_t* key,
                     uint64_t* u, size_t u_stride, int items, uint32_t g);
void launch_moddown_conv(he_ctx* c, const uint64_t* u, size_t u_stride, uint64_t* v,
                         size_t v_stride, int items);
void launch_ks_combine(he_ctx* c, const uint64_t* u, size_t u_stride, const uint64_t* v,
                       size_t v_stride, const uint64_t* const* c0p, const uint64_t* const* basep,
                       uint64_t* const* outp, int items, uint32_t g);
void launch_mac(he_ctx* c, const uint64_t* const* X, const uint64_t* const* P, int T,
                const uint64_t* const* accin, uint64_t* const* outp, int n_out, int L);
void launch_convpack(he_ctx* c, const uint64_t* x, int B, int r, int O_c, const uint64_t* wm,
                     uint64_t* const* outp, int L);
void launch_add(he_ctx* c, const uint64_t* const* a, const uint64_t* const* b,
                uint64_t* const* o, int items, int L);
// *bad |= 1 when a residue of `rows` rows (row r modulo mods[r % period]) is not below it.
void launch_check_range(he_ctx* c, const uint64_t* data, int rows, int period, int* bad);
// Pairs of polynomials over the first rows_per_poly moduli (e.g. Q u P): o = a + b.
void launch_add_rows(he_ctx* c, const uint64_t* const* a, const uint64_t* const* b,
                     uint64_t* const* o, int items, int rows_per_poly);
void launch_to_mont(he_ctx* c, uint64_t* data, int items, int rows, int period, int mod_off);
void launch_from_mont(he_ctx* c, uint64_t* data, int items, int rows, int period, int mod_off);
void launch_gather_last(he_ctx* c, const uint64_t* const* xp, uint64_t* last, int items, int L);
void launch_rescale_spread(he_ctx* c, const uint64_t* last, uint64_t* s, int items, int L);
void launch_rescale_combine(he_ctx* c, const uint64_t* const* xp, const uint64_t* s,
                            uint64_t* const* outp, int items, int L);
void launch_slots_to_ntt(he_ctx* c, const int64_t* v, uint64_t* buf, int items);
void launch_ntt_to_slots(he_ctx* c, const uint64_t* buf, int64_t* v, int items);
void launch_lift(he_ctx* c, const uint64_t* m, uint64_t* out, int items, int L, int mont);
void launch_from_signed(he_ctx* c, const int64_t* v, uint64_t* out, int rows, int mod_off);
void launch_uniform(he_ctx* c, uint64_t state0, uint64_t* out, int rows, int limb0, int mod_off);
void launch_gaussian(he_ctx* c, uint64_t state0, int64_t* out);
void launch_ternary(he_ctx* c, uint64_t state0, int64_t* out);
void launch_enc_c0(he_ctx* c, const int64_t* e, const uint64_t* m, const uint64_t* as,
                   const ShoupPair* delta, uint64_t* c0);
void launch_dec_phase(he_ctx* c, const uint64_t* ct, const uint64_t* s_m, uint64_t* x, int rows);
void launch_dec_round(he_ctx* c, const uint64_t* x, uint64_t* m, int L, int W,
                      const uint64_t* cst);

void launch_dec_phase_mul(he_ctx* c, uint64_t* x, const uint64_t* s_m, int rows);
void launch_keygen_b(he_ctx* c, const uint64_t* a, const uint64_t* s_m, const uint64_t* e,
                     const uint64_t* sg, uint64_t* b, int i0, int i1);

// layer kernels (layer.cu)
void launch_dp_shift_slots(he_ctx* c, const int32_t* w1, const he_layout& lay, int64_t* out);
void launch_dp_dot_slots(he_ctx* c, const int32_t* w1, const he_layout& lay, int64_t* out);
