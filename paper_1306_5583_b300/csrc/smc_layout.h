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
constexpr int kSelItems = 4;                    // outputs per thread, ancestor selection
constexpr int kSelTile = kBlock * kSelItems;    // 1024 outputs per block
constexpr int kSelCap = 2 * kScanTile;          // CDF entries staged in shared memory
constexpr int kMaxSplitters = 4096;             // scan tiles whose ends fit in shared memory
constexpr int kScanSlots = 6;                   // independent scans per iteration
constexpr uint32_t kSpinLimit = 1u << 24;       // bounded waits (about 1 s with backoff)

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
constexpr int SLOT_BUCKET = 1;   // bucket offsets of the uniform sort
constexpr int SLOT_RES_R = 2;    // residual-weight CDF
constexpr int SLOT_RES_O = 3;    // residual final offspring CDF

struct DevState {
    int32_t t;        // last completed iteration, -1 before initialize
    int32_t cur;      // which state buffer holds the current particles
    int32_t due;      // the ESS test of iteration t asked for resampling
    int32_t ready;    // ancestors for the next gather are in place
    int32_t error;    // device error word (SMC_E_*)
    int32_t pad_e;
    uint32_t ticket;  // last-block ticket of the weighting kernels
    uint32_t count_r; // residual: number of residual draws R
    double max_lw;    // M_t = max_i lw_t,i (the fixed-point shift)
    double log_norm;  // L_t
    double log_evidence;
    double ess;
    double alpha;     // GMM alpha_t
    double path_u;    // GMM U_t
    double path_log_z;
    double pad0;
    unsigned long long qn;     // fixed-point total of the last weight CDF
    unsigned long long sum_d;  // residual: sum of the deterministic copies
    uint32_t scan_counter[kScanSlots];  // tile ids handed out by a running scan
    uint32_t scan_done[kScanSlots];     // tiles finished by a running scan
    uint32_t scan_parity[kScanSlots];   // which status array a scan uses
    uint32_t accept[3];                 // GMM accepted moves per block (last mcmc)
    uint32_t pad1;
};

struct Partial {  // one per block of a weighting kernel
    double m, s1, s2, sx, sy, su;
    double pad[2];
};

// Tile status word of the decoupled look-back scans: bits 62-63 hold the
// status (1 = tile aggregate, 2 = inclusive prefix), bits 0-61 the value.
constexpr unsigned long long kStatAgg = 1ull << 62;
constexpr unsigned long long kStatIncl = 2ull << 62;
constexpr unsigned long long kStatMask = 3ull << 62;

struct ScanSlot {
    unsigned long long *status[2];  // [parity][tile]
    int32_t ntiles_max;
};

}  // namespace smc
