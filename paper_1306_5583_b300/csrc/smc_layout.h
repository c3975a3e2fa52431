// Shared host/device layout of the SMC context: device state word block,
// per-block reduction partials, kernel argument blocks and tile sizes.
#pragma once

#include <cstdint>

#include "../../include/smc.h"

namespace smc {

constexpr int kBlock = 256;                     // threads per block everywhere
constexpr int kPfItems = 4;                     // particles per thread, weighting kernels
constexpr int kPfTile = kBlock * kPfItems;      // 1024 particles per block
constexpr int kScanItems = 8;                   // elements per thread, scans
constexpr int kScanTile = kBlock * kScanItems;  // 2048 elements per scan tile
constexpr int kScanSlots = 6;                   // independent scans per iteration
constexpr uint32_t kSpinLimit = 1u << 24;       // bounded waits (about 1 s with backoff)

// Active threads per block of the double-precision particle filter's move
// tiles (one particle per thread): 64 for N <= 2^16, so that a small filter's
// float64 work spreads over many SMs, else every thread of the block.  The
// plain filter and the batched filters tile the same way (same partials,
// same normaliser).
__host__ __device__ constexpr int pf64_move_threads(int64_t n) { return n <= 65536 ? 64 : kBlock; }

// Histogram of the 24-bit multinomial draws: one byte count per value, four
// to a 32-bit word, 16 values (one uint4) to a bucket, kScanTile buckets to a
// histogram tile.
constexpr int kHistValueBits = 24;
constexpr int64_t kHistWords = int64_t(1) << (kHistValueBits - 2);
constexpr int64_t kHistBuckets = int64_t(1) << (kHistValueBits - 4);
constexpr int kHistTiles = (int)(kHistBuckets / kScanTile);  // 512

// Philox purpose tags (counter word 2, low 16 bits)
constexpr uint32_t TAG_INIT = 1;
constexpr uint32_t TAG_MOVE = 2;
constexpr uint32_t TAG_RESAMPLE = 3;
constexpr uint32_t TAG_MH_MU = 4;
constexpr uint32_t TAG_MH_LAMBDA = 5;
constexpr uint32_t TAG_MH_WEIGHT = 6;
constexpr uint32_t TAG_MALA = 7;
constexpr uint32_t DRAW_MH_UNIFORM = 16;

// scan slots
constexpr int SLOT_CDF = 0;      // fixed-point weight CDF
constexpr int SLOT_RES_D = 2;    // residual: tile sums of the deterministic copies
constexpr int SLOT_RES_R = 3;    // residual: tile sums of the residual weights

struct DevState {
    int32_t t;        // last completed iteration, -1 before initialize
    int32_t cur;      // which state buffer holds the current particles
    int32_t due;      // the ESS test of iteration t asked for resampling
    int32_t ready;    // ancestors for the next gather are in place
    int32_t error;    // device error word (SMC_E_*)
    int32_t cur_lw;   // which log-weight buffer is current
    uint32_t ticket;  // last-block ticket of the weighting kernels
    uint32_t pad1;
    double max_lw;    // M_t = max_i lw_t,i (the fixed-point shift)
    double log_norm;  // L_t
    double log_evidence;
    double ess;
    double alpha;     // GMM alpha_t
    double path_u;    // GMM U_t
    double path_log_z;
    double base_shift;  // log W_i = lw_i - base_shift (GMM; 0 after a gather resets lw to -log N)
    uint32_t scan_ticket[kScanSlots];   // last-block tickets of the tile-sum passes
    unsigned long long scan_total[kScanSlots];  // exact totals of the tile-sum passes
    uint32_t accept[4];                 // GMM accepted moves per block and Langevin (last mcmc)
    int32_t gathered;                   // GMM: the last mcmc gathered by ancestors
    int32_t pad2;
    float log_norm_f[2];  // L_t as an unevaluated float sum hi + lo (FP32 kernels)
    float max_lw_f;       // M_t as float (exact: the maximum of float log-weights)
    uint32_t grid_count;  // grid barrier of the one-pass resampling kernel: arrivals
    uint32_t grid_depart; // and departures (the last departure clears both)
    uint32_t pad3;
};

// Staging of smc_iterate_host in pinned host memory mapped into the device's
// address space: the device reads the step's observation and writes the
// step's record and error word through it (no separate copies).
struct HostIO {
    double obs[2];     // the observation of the next iteration (CV models)
    float obs_f[2];    // its float copy (the copy path without the graph)
    int32_t has_obs;   // 1: obs holds the next observation
    int32_t status;    // the device error word after the step
    smc_record rec;    // the step's record
    uint32_t done;     // the call's sequence number, written by the call's last kernel
    uint32_t pad;
};

struct Partial {  // one per block of a weighting kernel
    double m, s1, s2, sx, sy, su;
    double pad[2];
};


}  // namespace smc
