// ge_tb_plan.cpp -- host-side planning of the tiled kernel's launches, shared
// by the context API (ge_api.cpp) and ge_solve_noalloc (ge_noalloc.cu): the
// launch-independent coefficients of the right-hand-side form, and the loop
// that cuts a solve into launches and mirrors the kernel's scale recurrence.
// Host code only; built with -ffp-contract=off so the coefficients are
// rounded exactly as written.
#include <cmath>

#include "ge_internal.h"

namespace ge {

void tb_fill_base(double r, double beta_l, double beta_r, int prec, TbParams *out, double *growth_lo)
{
    TbParams p{};
    const double det = 1.0 + 2.0 * r;
    p.g = 2.0 * r;
    // The scaled block map x <- x + g x_partner multiplies the symmetric part
    // of every pair by exactly 1 + g, with g the coefficient the kernel holds
    // (rounded to FP32 on the FP32 path).  The host's scale mirror uses that
    // factor, carried as a double-double (onepg + growth_lo == 1 + g
    // exactly), so no systematic scale error builds up over many steps.
    scaled_growth(r, prec == 1, &p.onepg, growth_lo);
    p.stall = 0;
    p.emu = 1;
    p.r = r;
    p.omr = 1.0 - r;
    p.d = 2.0 * r / det;
    p.f_l = r * beta_l;
    p.f_r = r * beta_r;
    // exit u = ((1+r) w_i + r w_partner) / (1+2r); singleton w_i / (1+r)
    p.x1 = (1.0 + r) / det;
    p.x2 = r / det;
    p.xs = 1.0 / (1.0 + r);
    if (prec == 2) {
        p.kappa = (1.0 - r) / (1.0 + r);
        p.rescale_every = 0;
    } else {
        p.kappa = det * (1.0 - r) / (1.0 + r);
        // block steps between rescalings: the scale grows by (1+2r) per step
        // and stays below 2^headroom (data magnitudes up to 2^(max_exp -
        // headroom - 1) are safe)
        const double headroom = (prec == 0) ? kF64Headroom : GE_F32_HEADROOM;
        const int every = (int)std::floor(headroom / std::log2(1.0 + 2.0 * r));
        p.rescale_every = every < 1 ? 1 : every;
    }
    *out = p;
}

int tb_clamp_depth(const TbParams &base, int depth)
{
    const int every = base.rescale_every;
    if (every > 0 && depth > (kMaxRescale - 1) * every)
        depth = (kMaxRescale - 1) * every;
    if (depth > kMaxTableSteps)
        depth = kMaxTableSteps;
    return depth;
}

cudaError_t tb_run(const TbTarget &t, const TbParams &base, double growth_lo, bool df, int prec, int *cur,
                   long long step0, long long steps, int depth, cudaStream_t s)
{
    depth = tb_clamp_depth(base, depth);
    if (depth < 1)
        return cudaErrorInvalidValue;
    const int every = base.rescale_every;
    double sigma = 1.0, sigma_lo = 0.0;  // double-double scale
    int until = every;
    long long n0 = 0;
    // the tiled launches' queue words: both zero now; each launch zeroes the
    // one the next launch uses
    int k_tiled = 0;
    if (steps > 0) {
        const cudaError_t e = cudaMemsetAsync(t.tile_ctr, 0, 2 * sizeof(int), s);
        if (e != cudaSuccess)
            return e;
    }
    while (n0 < steps) {
        const long long L = (steps - n0 < depth) ? steps - n0 : depth;
        TbParams p = base;
        const bool last = (n0 + L == steps);
        p.do_entry = (n0 == 0) ? 1 : 0;
        p.n_mid = (int)(last ? L - 1 : L);
        p.do_exit = last ? 1 : 0;
        p.p_first = (int)((step0 + n0) & 1);
        p.sigma_in = sigma;
        p.rescale_phase = until;
        if (every > 0) {
            int ev = 0;
            for (int m = 0; m < p.n_mid; ++m) {
                dd_mul(sigma, sigma_lo, p.onepg, growth_lo);
                if (--until == 0) {
                    until = every;
                    int e2 = 0;
                    std::frexp(sigma, &e2);
                    const int e = e2 - 1;  // sigma * 2^-e in [1, 2)
                    p.rs_exp[ev++] = (short)e;
                    sigma = std::ldexp(sigma, -e);
                    sigma_lo = std::ldexp(sigma_lo, -e);
                }
            }
        }
        if (p.do_exit) {
            p.x1 = dd_div(base.x1, sigma, sigma_lo);
            p.x2 = dd_div(base.x2, sigma, sigma_lo);
            p.xs = dd_div(base.xs, sigma, sigma_lo);
            df_split_host(p.x1, p.dfc[4]);
            df_split_host(p.x2, p.dfc[5]);
            df_split_host(p.xs, p.dfc[6]);
        }
        p.df_in = p.do_entry;
        p.df_out = p.do_exit;
        const int reach = p.do_entry + p.n_mid + p.do_exit;
        if (!(df ? tb_df_geometry(reach, &p.H, &p.U) : tb_geometry(prec, reach, &p.H, &p.U)))
            return cudaErrorInvalidValue;
        p.n = t.n;
        p.n_rows = t.n_rows;
        p.n_tiles = (t.n + p.U - 1) / p.U;
        p.out = t.buf[*cur ^ 1];
        p.err = t.err;
        p.tile_ctr = t.tile_ctr + (k_tiled & 1);
        p.tile_ctr_next = t.tile_ctr + ((k_tiled + 1) & 1);
        long long grid = t.grid_cap;
        if (grid > p.n_tiles)
            grid = p.n_tiles;
        if (grid < 1)
            grid = 1;
        cudaError_t e;
        if (!df && prec == 1 && p.n_mid == 1 && !p.do_entry && !p.do_exit && p.stall == 0) {
            // one FP32 block step and nothing else: an HBM stream, no tiles
            e = launch_tb_stream(prec, t.buf[*cur], p.out, p, s);
        } else {
            e = df ? launch_tb_df(t.tmap[*cur], p, (int)grid, s) : launch_tb(prec, t.tmap[*cur], p, (int)grid, s);
            ++k_tiled;
        }
        if (e != cudaSuccess)
            return e;
        *cur ^= 1;
        n0 += L;
    }
    return cudaSuccess;
}

}  // namespace ge
