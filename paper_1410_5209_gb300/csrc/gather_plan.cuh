// Gather plan of the lean float pass: the step records the pass walks and the location
// word of every entry (built by gather_plan.cu, read by lean_pass.cu).
#pragma once

#include "common.cuh"

namespace tfs {

// Location words: bit 15 marks a staging-pool position (else a cache row); kKeep in the
// run-mode half says the lane already holds the products of that row.
constexpr uint32_t kPoolBit = 0x8000u, kKeep = 0xFFFFu;

// Step record of a gather plan: lanes [lo, hi) of the 32-entry step starting at entry j0
// of one item (a step's lanes are split over several records when its distinct cold rows
// exceed the pool; each lane still takes the same entry as in an unsplit step, so the
// per-lane sums, and the results, do not depend on the split).  info packs hi (bits 0-5),
// first record of the item (6), last record of the item (7), own-row buffer (8-9), staged
// varying-mode rows nV (10-15), run-mode rows nR (16-21) and lo (22-26); the record's cold
// rows are list[list_off .. + nV + nR) (varying first).
struct GStep {
    int32_t j0;
    uint32_t list_off;
    uint32_t info;
    int32_t slot;  // partial slot of the item
};

// Records one 32-entry step can take with a pool of cap >= 2 rows: every record but the
// last of a step holds at least cap - 1 of the step's at most 64 cold rows (a lane adds at
// most two), and every record at least one lane.
__host__ __device__ constexpr int plan_records_per_step(int cap) {
    return 64 / (cap - 1) + 1 < 32 ? 64 / (cap - 1) + 1 : 32;
}

}  // namespace tfs
