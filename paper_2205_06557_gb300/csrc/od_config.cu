// Pair-kernel configuration of a run: the autotuner (od_tune), a known choice
// (od_set_force_config / od_get_force_config) and the ion-ion cutoff (od_set_cutoff).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "od_host.h"

using namespace od;
using namespace od::host;

namespace od {
namespace host {

static const int kTuneGrains[4] = {4, 8, 16, 32};
static const int kTuneBps[3] = {0, 4, 2};  // persistent CTAs per SM: 0 = occupancy limit

// close-pair correction on when the FP32 ion-ion kernels run, and under the cutoff only
// while the correction distance lies inside the plain (unswitched) zone
void set_close_pairs(od_handle* h)
{
    const double ls = 1.4426950408889634 * h->P.lam_inv;
    h->P.cp_on = !(h->P.flags & (OD_F_NO_IONION | OD_F_FP64_PAIRS)) &&
                 (!h->cut_on || h->r_switch * ls * h->r_switch * ls >= h->P.cp_dc2);
}

int apply_force_config(od_handle* h, int variant, int upb, int bps)
{
    h->variant = variant;
    h->upb = upb;
    h->bps = bps;
    int rc = replan(h, h->P.N);
    if (rc) return rc;
    h->graph_ok = false;
    // the padded length may have grown: rewrite positions and far-away dummies
    OD_LK(h, launch_fpos(h->P, h->B, (int)(h->host_step & 1), h->stream));
    return OD_OK;
}

}  // namespace host
}  // namespace od

extern "C" {

int od_set_cutoff(od_handle* h, double r_cut, double r_switch)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (h->batch_member) return fail(h, OD_EINVAL, "the cutoff is set on single runs, not batch members");
    if (h->P.flags & OD_F_FLUX_INJECT) return fail(h, OD_EINVAL, "the cutoff needs a fixed ion count (no flux rule)");
    if (h->P.flags & OD_F_FP64_PAIRS) return fail(h, OD_EINVAL, "the cutoff runs on the FP32 kernels only");
    if (!std::isfinite(r_cut) || !std::isfinite(r_switch)) return fail(h, OD_EINVAL, "cutoff: non-finite distance");
    OD_CK(h, cudaStreamSynchronize(h->stream));
    int rc;
    if (r_cut <= 0.0) {
        if (!h->cut_on) return OD_OK;
        h->cut_on = false;
        h->r_cut = h->r_switch = 0.0;
        free_cut(h);
        set_close_pairs(h);
        if ((rc = replan(h, h->P.N))) return rc;
        h->graph_ok = false;
        if ((rc = force_eval(h))) return rc;
        OD_CK(h, cudaStreamSynchronize(h->stream));
        return read_error_word(h);
    }
    if (!(r_switch >= 0.0 && r_switch < r_cut)) return fail(h, OD_EINVAL, "cutoff: need 0 <= r_switch < r_cut");
    constexpr int TI = 512;
    const long long npad_max = (h->cap + TI - 1) / TI * TI;
    const int T = (int)(npad_max / TI);
    if (T > CUT_MAX_TILES)
        return fail(h, OD_EINVAL, "cutoff: at most " + std::to_string(CUT_MAX_TILES * TI) + " ions");
    // slabs of about an eighth of the cutoff (the slab-by-warp count matrix stays below
    // 64M entries)
    const long long nblk = (h->cap + 31) / 32;
    int nslab = (int)std::min(65536.0, std::max(1.0, std::ceil(h->P.H / (r_cut / 8.0))));
    while ((long long)nslab * nblk > (64ll << 20) && nslab > 1) nslab = (nslab + 1) / 2;
    const double w = h->P.H / nslab;
    free_cut(h);
    CutBufs& C = h->C;
    const double ls = 1.4426950408889634 * h->P.lam_inv;
    C.nslab = nslab;
    C.zoff = (float)(0.5 * h->P.H * ls);
    C.inv_w = (float)(1.0 / (w * ls));
    const double rcs = r_cut * ls * (1.0 + 1e-5);  // box test: never drop a pair inside the cutoff
    C.rc2_tile = (float)(rcs * rcs);
    const double rss = r_switch * ls * (1.0 - 1e-5);  // plain units: never skip a switched pair
    C.rs2_tile = (float)(rss * rss);
    const long long M = (long long)nslab * nblk;
    const long long nchunk = (M + 8191) / 8192;
    OD_CK(h, cudaMalloc(&C.bcount, sizeof(int) * M));
    OD_CK(h, cudaMalloc(&C.boff, sizeof(int) * M));
    OD_CK(h, cudaMalloc(&C.bsum, sizeof(int) * nchunk));
    OD_CK(h, cudaMalloc(&C.perm, sizeof(int) * h->cap));
    OD_CK(h, cudaMalloc(&C.rank, sizeof(int) * h->cap));
    OD_CK(h, cudaMalloc(&C.fsort, sizeof(float4) * npad_max));
    OD_CK(h, cudaMalloc(&C.box_lo, sizeof(float4) * T));
    OD_CK(h, cudaMalloc(&C.box_hi, sizeof(float4) * T));
    OD_CK(h, cudaMalloc(&C.units, sizeof(int2) * ((size_t)T * (T + 1) / 2)));
    OD_CK(h, cudaMalloc(&C.n_units, sizeof(int)));
    OD_CK(h, cudaMalloc(&C.ucnt, sizeof(int) * T));
    OD_CK(h, cudaMalloc(&C.ustart, sizeof(int) * T));
    h->cut_on = true;
    h->r_cut = r_cut;
    h->r_switch = r_switch;
    h->cut_grid = h->sms * cut_blocks_per_sm(2);
    set_close_pairs(h);
    if ((rc = replan(h, h->P.N))) return rc;
    OD_LK(h, launch_cut_dummies(C, h->P.N, h->F.n_pad, h->stream));
    h->graph_ok = false;
    if ((rc = force_eval(h))) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    return read_error_word(h);
}



int od_set_force_config(od_handle* h, int variant, int units_per_block, int blocks_per_sm)
{
    if (!h || variant < 0 || variant >= num_force_variants() || units_per_block < 1 || units_per_block > 1024 ||
        blocks_per_sm < 0 || blocks_per_sm > 64 || h->batch_member)
        return fail(h, OD_EINVAL, "bad force configuration (or a batch member: use od_batch_set_config)");
    int rc = apply_force_config(h, variant, units_per_block, blocks_per_sm);
    if (rc) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    return OD_OK;
}

int od_tune(od_handle* h, int reps, double* ms, int* best_variant, int* best_upb, int* best_bps)
{
    if (!h || reps < 1 || h->batch_member)
        return fail(h, OD_EINVAL, "bad handle or repetition count (or a batch member: use od_batch_tune)");
    if (h->cut_on) return fail(h, OD_EINVAL, "the cutoff has a fixed plan: switch it off to tune the all-pairs kernels");
    if (h->P.flags & OD_F_FP64_PAIRS) return fail(h, OD_EINVAL, "the FP64 study kernel has no variants to tune");
    const int nv = num_force_variants();
    if (ms)
        for (int i = 0; i < nv * 4 * 3; ++i) ms[i] = -1.0;
    if (h->P.N == 0 || (h->P.flags & OD_F_NO_IONION)) {
        if (best_variant) *best_variant = h->variant;
        if (best_upb) *best_upb = h->upb;
        if (best_bps) *best_bps = h->bps;
        return OD_OK;
    }
    double best = 1e300;
    int bv = h->variant, bg = h->upb, bb = h->bps;
    struct Timed {
        double ms;
        int v, g, b;
    };
    std::vector<Timed> timed;
    for (int v = 0; v < nv; ++v)
        for (int g = 0; g < 4; ++g)
            for (int c = 0; c < 3; ++c) {
                if (kTuneBps[c] >= force_blocks_per_sm(v)) continue;  // no cap below the occupancy limit
                const ForceVariant fv = force_variant(v);
                if (fv.sym && g > 0) continue;  // fixed-size units: one grain setting
                int rc = apply_force_config(h, v, kTuneGrains[g], kTuneBps[c]);
                if (rc) return rc;
                // the kick is timed too: it sums the ordered kernel's partial slots, or reads
                // and clears the symmetric kernels' fixed-point sums
                OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
                OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
                OD_CK(h, cudaEventRecord(h->ev[0], h->stream));
                for (int r = 0; r < reps; ++r) {
                    OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
                    OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
                }
                OD_CK(h, cudaEventRecord(h->ev[1], h->stream));
                OD_CK(h, cudaEventSynchronize(h->ev[1]));
                float t = 0.f;
                OD_CK(h, cudaEventElapsedTime(&t, h->ev[0], h->ev[1]));
                const double avg = t / reps;
                if (ms) ms[(v * 4 + g) * 3 + c] = avg;
                timed.push_back({avg, v, kTuneGrains[g], kTuneBps[c]});
            }
    // final round: the three fastest settings again, in turn, three times each, so that a
    // difference of a few percent is not decided by one noisy sample
    std::sort(timed.begin(), timed.end(), [](const Timed& a, const Timed& b) { return a.ms < b.ms; });
    const int nf = (int)std::min<size_t>(3, timed.size());
    std::vector<double> total(nf, 0.0);
    for (int round = 0; round < 3 && nf > 1; ++round)
        for (int f = 0; f < nf; ++f) {
            int rc = apply_force_config(h, timed[f].v, timed[f].g, timed[f].b);
            if (rc) return rc;
            OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
            OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
            OD_CK(h, cudaEventRecord(h->ev[0], h->stream));
            for (int r = 0; r < reps; ++r) {
                OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
                OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
            }
            OD_CK(h, cudaEventRecord(h->ev[1], h->stream));
            OD_CK(h, cudaEventSynchronize(h->ev[1]));
            float t = 0.f;
            OD_CK(h, cudaEventElapsedTime(&t, h->ev[0], h->ev[1]));
            total[f] += t;
        }
    for (int f = 0; f < nf; ++f)
        if (f == 0 || total[f] < best) {
            best = total[f];
            bv = timed[f].v;
            bg = timed[f].g;
            bb = timed[f].b;
        }
    int rc = apply_force_config(h, bv, bg, bb);
    if (rc) return rc;
    // give back partial-slot memory beyond what the chosen layout needs
    if (h->part_cap > 2 * (long long)h->F.W * h->F.n_pad && h->part_cap > 0) {
        OD_CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->B.part);
        h->B.part = nullptr;
        h->part_cap = 0;
        if ((rc = ensure_part(h))) return rc;
    }
    // the accelerations and partial sums left by the timing belong to other kernels:
    // evaluate the current state again with the chosen one
    if ((rc = force_eval(h))) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    if (best_variant) *best_variant = bv;
    if (best_upb) *best_upb = bg;
    if (best_bps) *best_bps = bb;
    return read_error_word(h);
}

int od_get_force_config(od_handle* h, int* variant, int* units_per_block, int* blocks_per_sm, int* n_variants)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (variant) *variant = h->variant;
    if (units_per_block) *units_per_block = h->upb;
    if (blocks_per_sm) *blocks_per_sm = h->bps;
    if (n_variants) *n_variants = num_force_variants();
    return OD_OK;
}


}  // extern "C"
