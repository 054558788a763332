// eval.cuh -- rotation / MAC / rescale building blocks shared by the entry points and the layer.
#pragma once

#include <vector>

#include "he_internal.cuh"

struct RotBufs {
    uint64_t* T;   // [items][L][N]        c1 (after the automorphism) in coefficient form
    uint64_t* D;   // [items][dnum][L+K][N] ModUp digits, NTT domain
    uint64_t* u;   // [items][2][L+K][N]   key inner products
    uint64_t* v;   // [items][2][L][N]     ModDown base conversions
};

size_t rot_scratch_per_item(const he_ctx* c);
RotBufs rot_bufs_take(he_ctx* c, int items);
void modup_items(he_ctx* c, const uint64_t* X, int items, uint32_t g_own, const RotBufs& b);
void moddown_items(he_ctx* c, uint64_t* u, uint64_t* v, int items);
void moddown_combine(he_ctx* c, uint64_t* u, uint64_t* v, int items, const uint64_t* const* c0p,
                     const uint64_t* const* basep, uint64_t* const* outp, uint32_t g);
void ks_items(he_ctx* c, int items, const uint64_t* key, uint32_t g_ks, uint32_t g,
              const uint64_t* const* c0p, const uint64_t* const* basep, uint64_t* const* outp,
              const RotBufs& b);
const uint64_t* const* upload_ptrs(he_ctx* c, const std::vector<const uint64_t*>& v);
uint64_t* const* upload_out_ptrs(he_ctx* c, const std::vector<uint64_t*>& v);
int rotate_contig(he_ctx* c, const uint64_t* X, int items, uint32_t g, const uint64_t* base,
                  const std::vector<uint64_t*>& outs, const RotBufs& b, int chunk);
int rotate_hoisted_contig(he_ctx* c, const uint64_t* X, int items, const std::vector<uint32_t>& gs,
                          const std::vector<uint64_t*>& outs, const RotBufs& b);
int rotation_chunk(const he_ctx* c);
int max_mac_terms(const he_ctx* c);
int rescale_items(he_ctx* c, const std::vector<const uint64_t*>& xs,
                  const std::vector<uint64_t*>& outs, int Lv, uint64_t* last, uint64_t* s);
int he_key_for_generation(he_ctx* ctx, uint32_t g, uint64_t** dev);
