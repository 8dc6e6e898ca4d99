// Batched launch of many instances (internal; see batch.cu).
#pragma once

#include "lbm_kernels.h"

namespace pwfa {

constexpr int kBatchTile = 128;     // consecutive nodes (threads) per fluid work tile
// consecutive fluid tiles of one instance per block of the per-node phases
// (the block's set-up: its instance, the argument copy, is paid once per
// group)
#ifndef PWFA_BATCH_TILES
#define PWFA_BATCH_TILES 2
#endif
constexpr int kBatchGroup = PWFA_BATCH_TILES;
constexpr int kMaxBatch = 65535;    // instances per batched launch (16-bit block -> instance map)

// One instance of the batch, in device memory.
struct BatchEntry {
    StepArgs args[2];     // step arguments for the two ping-pong parities
    FieldPair out[2];     // the fused field step's outputs for the two parities
    int64_t tile_begin;   // first block (group of kBatchGroup fluid tiles) of the instance
    int64_t ntiles;       // fluid tiles of the instance
    int64_t ftile_begin;  // first fused-field tile
    int ftiles_x, ftiles_y;  // fused-field tiles per z-slab
    double z0, dt;        // driver centre at t = 0 and time step
    int64_t* step;        // two device step counters: the step index n of the
                          // step that the launches of parity p take is
                          // step[p]; each Ampere (or fused field) launch of
                          // parity p writes step[p ^ 1] = step[p] + 1, so the
                          // replayed graph advances its own driver time
};

struct BatchLaunch {
    const BatchEntry* entries;         // device copy of the table
    const uint16_t* tile_inst;         // instance of each block of fluid tiles
    const uint16_t* ftile_inst;        // instance of each fused-field tile
    int ninst;
    int64_t ntiles, nftiles;           // blocks of the per-node phases, fused-field tiles
};

// Phases of one batched step: 0 Faraday, 1 fluid, 2 Ampere (per-node, on
// the fluid tiles), 3 Ampere fused with the next step's Faraday (on the
// fused-field tiles), each one launch over every instance.
cudaError_t launch_batch_phase(const BatchLaunch& b, int phase, int parity, int storage, int collision,
                               bool periodic, cudaStream_t s);

}  // namespace pwfa
