// graph.h -- internal interface between the C ABI (ecmc.cu) and the
// constraint-graph path (graph.cu, ECMC_GRAPH). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ecmc.h"

struct GraphCtx;

// Totals of one graph_run call.
struct GraphTotals {
    int64_t legs, lifts, conflict_legs, repaired, continued, horizon, order_err, p1_lifts,
        repair_lifts, restarts, blocked, cwindows;
    double ms, pass1_ms, repair_ms, other_ms;
};

// A context on device inputs x, y (n each) and active (k), all device
// pointers valid until the call returns; nc cells per side are used only to
// build the graph.
int graph_create(const ecmc_params *p, int nc, const double *x, const double *y,
                 const int32_t *active, cudaStream_t st, GraphCtx **out, std::string &err);
int graph_run(GraphCtx *g, int32_t n_legs, uint64_t budget, uint8_t *flags_host,
              int32_t *legs_done, GraphTotals *tot, std::string &err);
// Device outputs (each may be null), filled on the context's stream.
int graph_export(GraphCtx *g, double *x, double *y, double *t, int32_t *active);
// Exchanges x and y of every disk (the next legs move along the other axis),
// clears the local times and rebuilds the graph.
int graph_transpose(GraphCtx *g, std::string &err);
// Host copies of the arrows (3 per disk, -1: none) and their b_ij.
int graph_arrows(GraphCtx *g, int32_t *a, double *b, std::string &err);
int graph_liftings(GraphCtx *g, ecmc_lift_t *buf, int64_t cap, int64_t *n_out,
                   std::string &err);
void graph_destroy(GraphCtx *g);
// Batches of graph contexts: one persistent launch advances n contexts (same
// claim windows, no restart mode), each to max_legs legs or its liftings
// budget (budgets may be null; 0: none), exactly as graph_run would. The
// scratch (launch tables) is kept by the caller between calls and freed with
// graph_batch_free. tots[r] and legs_out[r] (may be null) receive each
// context's totals; *ms_out the launch's device time.
struct GBatchScratch;
int graph_batch_run(GBatchScratch **scratch, GraphCtx *const *gs, int32_t n, int32_t max_legs,
                    const uint64_t *budgets, cudaStream_t st, GraphTotals *tots,
                    int32_t *legs_out, double *ms_out, std::string &err);
void graph_batch_free(GBatchScratch *scratch);
// Device memory held by the context (bytes).
int64_t graph_device_bytes(const GraphCtx *g);
// What graph_create(p, nc, ...) would hold, without allocating (-1: error).
int64_t graph_plan_bytes(const ecmc_params *p, int nc);
