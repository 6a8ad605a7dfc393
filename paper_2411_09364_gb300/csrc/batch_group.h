// Grouped execution of a batch of FP32 + refinement solves (internal).
//
// Every solve of the batch runs the same stages (forward x, y, z, inverse y,
// x; per refinement sweep a residual and the same five stages).  Instead of
// one launch per stage per solve, each stage of all solves is one launch (or
// a few, one per kernel variant): CTA b of the launch looks up its (solve,
// block) pair in a work list and the solve's argument block in device memory.
#pragma once
#include <vector>

#include "cales.h"
#include "plan.h"

struct GroupedBatch;

// Build the argument blocks and work lists of every stage for the buffers
// f[i] -> u[i] (uploaded with synchronous copies; call outside stream
// capture).  Returns nullptr with *rc = CALES_OK when the batch does not
// qualify (precision other than FP32 + refinement, unequal sweep counts, a
// periodic z, a plan used by two solves, a z line that does not take the
// warp-per-segment kernel); nullptr with *rc < 0 on error.
GroupedBatch* grouped_build(const std::vector<cales_plan_t>& plans, const std::vector<int>& kinds,
                            const std::vector<double>& alphas, const void* const* f, void* const* u, int* rc);
// True when the batch was built for exactly these buffers.
bool grouped_same_buffers(const GroupedBatch* g, const void* const* f, void* const* u);
// Enqueue every stage on one stream (graph-capturable).
int grouped_enqueue(GroupedBatch* g, cudaStream_t st);
// Launches per enqueue (kernels and memsets).
int grouped_launches(const GroupedBatch* g);
void grouped_free(GroupedBatch* g);
