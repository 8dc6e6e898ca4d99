// Batched persistent launch of many instances (internal; see batch.cu).
#pragma once

#include "lbm_kernels.h"

namespace pwfa {

constexpr int kBatchTile = 128;  // nodes (threads) per work item
constexpr int kMaxBatch = 96;    // instances per batched launch (constant-memory table)
constexpr int kBatchCounters = 3; // work counters of the Faraday, fluid and Ampere phases

// One instance of the batch, in device memory.
struct BatchEntry {
    StepArgs args[2];    // step arguments for the two ping-pong parities
    int64_t item_begin;  // index of the instance's first work item
    int tiles_x, tiles_y;
    int bx, by;          // tile shape, bx * by = kBatchTile
    double z0, dt;       // driver centre at t = 0 and time step
    int64_t* step;       // device step counter (driver time t_{n+1} = (step + 1) dt)
};

struct BatchLaunch {
    const BatchEntry* entries;
    int ninst;
    int64_t nitems;
    int grid;            // persistent CTAs (SMs x resident blocks)
    int* counters;       // kBatchCounters work counters, zero before each phase
                         // (re-armed by the step-counter kernel)
};

// One phase of a step of every instance: 0 Faraday, 1 fluid, 2 Ampere,
// 3 advance the step counters and re-arm the work counters.
cudaError_t launch_batch_phase(const BatchLaunch& b, int phase, int parity, int storage, int collision,
                               bool periodic, cudaStream_t s);

// Copy the instance table into the kernels' constant-memory copy.
cudaError_t batch_upload_table(const BatchEntry* host, int n, cudaStream_t s);

// Persistent grid size for the given kernel variant.
cudaError_t batch_grid_size(int storage, int collision, bool periodic, int* grid);

}  // namespace pwfa
