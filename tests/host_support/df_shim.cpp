// Host build of the library's double-float and grid-threshold helpers, for
// the CPU tests (plain C entry points over the header-only code).
#include "../../paper_1306_5583_b300/csrc/df_math.h"
#include "../../paper_1306_5583_b300/csrc/grid_threshold.h"

extern "C" {
void shim_df_log(float hi, float lo, float *out) {
    const smc::DF r = smc::df_log(smc::DF{hi, lo});
    out[0] = r.hi;
    out[1] = r.lo;
}
void shim_df_div(float ah, float al, float bh, float bl, float *out) {
    const smc::DF r = smc::df_div(smc::DF{ah, al}, smc::DF{bh, bl});
    out[0] = r.hi;
    out[1] = r.lo;
}
double shim_df_to_double(float hi, float lo) { return smc::df_to_double(smc::DF{hi, lo}); }
void shim_df_from_u64(unsigned long long x, float *out) {
    const smc::DF r = smc::df_from_u64(x);
    out[0] = r.hi;
    out[1] = r.lo;
}
void shim_df_from_int(long long x, float *out) {
    const smc::DF r = smc::df_from_int(x);
    out[0] = r.hi;
    out[1] = r.lo;
}
// thresholds tau_{k0 + j}, j < count, with a constant c: per-k form
// (incremental = 0, as for stratified targets) or the advancing remainder
// form of systematic targets (incremental = 1)
void shim_grid_tau(unsigned long long qn, unsigned long long n, unsigned long long k0, unsigned long long c,
                   int count, int incremental, unsigned long long *out) {
    smc::GridDiv d;
    d.init(qn, n, ~0ull / n);
    uint64_t u, v;
    d.start(k0, u, v);
    uint64_t rem = 0, t = 0;
    for (int j = 0; j < count; ++j) {
        if (incremental) {
            if (j == 0) t = d.tau(k0, c, u, v, &rem);
            else d.advance(t, rem);
            out[j] = t;
        } else {
            if (j > 0) d.next(u, v);
            out[j] = d.tau(k0 + j, c, u, v);
        }
    }
}
}
