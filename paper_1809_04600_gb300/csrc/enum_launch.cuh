// Host-side launch helpers for the pair enumeration kernels (enumerate.cuh).
#pragma once
#include "context.cuh"
#include "enumerate.cuh"

namespace shci {

inline EnumArgs enum_args(const shci_ctx *c) {
    EnumArgs A{};
    A.dets = c->dets.p;
    A.astr = c->astr.p;
    A.bstr = c->bstr.p;
    A.ga_off = c->ga_off.p;
    A.gb_off = c->gb_off.p;
    A.ga_det = c->ga_det.p;
    A.gb_det = c->gb_det.p;
    A.ga_str = c->ga_str.p;
    A.gb_str = c->gb_str.p;
    A.as_off = c->as_off.p;
    A.as_idx = c->as_idx.p;
    A.work_counter = c->counter.p + 1;
    A.opp_lookup = c->opp_lookup ? 1 : 0;
    A.opp_hybrid = c->opp_hybrid ? 1 : 0;
    A.opp_factor = c->opp_factor;
    A.ib = c->ib.p;
    A.bs_off = c->bs_off.p;
    A.bs_idx = c->bs_idx.p;
    A.occ = c->occ.p;
    A.occ_pref = c->occ_pref.p;
    A.occ_words = c->occ_words;
    return A;
}

// One pass of the alpha-grouped (alpha_part) or beta-grouped enumeration:
// a persistent grid whose CTAs take work items from an atomic counter.
template <int W, int MODE, int K>
void launch_enum(shci_ctx *c, EnumArgs A, const DevInts &I, bool alpha_part) {
    CUDA_TRY(cudaMemsetAsync(c->counter.p + 1, 0, sizeof(int), c->st));
    if (!A.item_group) {                    // the context's items unless the caller gave its own
        A.item_group = alpha_part ? c->item_a_group.p : c->item_b_group.p;
        A.item_first = alpha_part ? c->item_a_first.p : c->item_b_first.p;
        A.n_items = alpha_part ? c->n_items_a : c->n_items_b;
    }
    const int blocks = c->n_sm * (2048 / ENUM_THREADS);
    if (alpha_part) k_enum_alpha<W, MODE, K><<<blocks, ENUM_THREADS, 0, c->st>>>(A, I);
    else k_enum_beta<W, MODE, K><<<blocks, ENUM_THREADS, 0, c->st>>>(A, I);
    KERNEL_CHECK();
    g_kernel_launches += 1;
}

}  // namespace shci
