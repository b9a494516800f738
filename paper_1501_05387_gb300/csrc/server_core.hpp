// Host-only core of the query server: admission of queued requests under a
// device-memory budget, batch formation, and the life cycle of one batch on
// a worker slot. No CUDA here: server.cu supplies the device side, and a
// CPU test drives the same code with a fake device.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <unordered_map>
#include <vector>

#include "gr.h"

namespace gr {
namespace serve {

// Scratch a slot keeps per graph, one kind per way of running a batch.
enum WsKind : int { kWsBfs = 0, kWsBfsBatch, kWsSssp, kWsSsspBatch, kWsCc, kWsKinds };

inline WsKind ws_kind(int32_t query_kind, bool many) {
  if (query_kind == GR_QUERY_BFS) return many ? kWsBfsBatch : kWsBfs;
  if (query_kind == GR_QUERY_SSSP) return many ? kWsSsspBatch : kWsSssp;
  return kWsCc;
}

struct GraphInfo {
  int32_t n = 0;
  // a BFS request runs as a lane of a batch once at least this many BFS
  // requests for the graph are queued (0: never batched)
  int32_t min_batch = 1;
  // most SSSP requests one batched search takes (1: never batched)
  int32_t sssp_lanes = 1;
  size_t ws_bytes[kWsKinds] = {};   // what creating each workspace costs
  bool have_ws[kWsKinds] = {};      // created by the slot (kept until exit)
};

struct Pending {
  int32_t graph = 0;
  int32_t kind = 0;
};

// Admission and batching state (the caller serialises access). A batch
// holds requests of one kind on one graph. Device memory the server
// accounts for: the result buffers of the batch in flight (4n bytes per
// request) plus the workspaces the slot has created, which it keeps. A
// batch is admitted when what it adds (its result buffers and any
// workspace it must create) fits in the budget next to that; the oldest
// queued request is admitted alone even when it does not fit and nothing
// is in flight, so the queue always moves (the budget then bounds
// batching, not the one request).
struct Admission {
  size_t budget = 0;
  size_t in_use = 0;    // result buffers of the admitted, unfinished batch
  size_t resident = 0;  // workspaces created so far
  int32_t max_batch = 64;
  std::vector<GraphInfo> graphs;
  std::deque<uint64_t> queue;                     // tickets, arrival order
  std::unordered_map<uint64_t, Pending> pending;  // queued tickets

  size_t result_bytes(int32_t graph) const { return sizeof(int32_t) * (size_t)graphs[graph].n; }

  // result buffers a batch of `lanes` requests of `kind` holds: one per
  // request, except that the CC requests of a batch (all of one graph) share
  // one run and its one result
  static size_t result_units(int32_t kind, size_t lanes) {
    return kind == GR_QUERY_CC ? 1 : lanes;
  }

  // bytes a batch of `lanes` requests of `kind` on `graph` adds
  size_t cost(int32_t graph, int32_t kind, size_t lanes) const {
    const GraphInfo &gi = graphs[graph];
    const WsKind w = ws_kind(kind, lanes > 1);
    return result_units(kind, lanes) * result_bytes(graph) + (gi.have_ws[w] ? 0 : gi.ws_bytes[w]);
  }
  bool fits(size_t add) const { return resident + in_use + add <= budget; }

  // Most lanes a batch led by a request of `kind` on `graph` may take.
  int32_t lane_cap(int32_t graph, int32_t kind) const {
    const GraphInfo &gi = graphs[graph];
    if (max_batch <= 1 || gi.min_batch <= 0) return 1;
    if (kind == GR_QUERY_BFS) {
      int32_t queued = 0;  // the leader and the same-graph BFS requests behind it
      for (uint64_t t : queue) {
        const Pending &p = pending.at(t);
        if (p.kind == GR_QUERY_BFS && p.graph == graph && ++queued >= gi.min_batch) break;
      }
      return queued >= gi.min_batch ? max_batch : 1;
    }
    if (kind == GR_QUERY_SSSP) return std::min(max_batch, gi.sssp_lanes);
    return max_batch;  // CC: every queued request of the graph shares the run
  }

  // Next batch (tickets) for a free slot, or empty when the queue is empty
  // or the oldest request must wait for memory. Marks the batch admitted.
  std::vector<uint64_t> take_batch() {
    std::vector<uint64_t> out;
    if (queue.empty()) return out;
    const Pending lead = pending.at(queue.front());
    const int32_t cap = lane_cap(lead.graph, lead.kind);
    // the leader and the same-kind, same-graph requests behind it, up to cap
    std::vector<size_t> pos;
    for (size_t i = 0; i < queue.size() && (int32_t)pos.size() < cap; ++i) {
      const Pending &p = pending.at(queue[i]);
      if (p.kind == lead.kind && p.graph == lead.graph) pos.push_back(i);
    }
    // as many lanes as fit; a batched workspace that does not fit falls
    // back to the single one
    size_t lanes = pos.size();
    while (lanes > 1 && !fits(cost(lead.graph, lead.kind, lanes))) --lanes;
    if (!fits(cost(lead.graph, lead.kind, lanes)) && in_use > 0) return out;  // wait
    pos.resize(lanes);
    GraphInfo &gi = graphs[lead.graph];
    const WsKind w = ws_kind(lead.kind, lanes > 1);
    if (!gi.have_ws[w]) {
      gi.have_ws[w] = true;
      resident += gi.ws_bytes[w];
    }
    in_use += result_units(lead.kind, lanes) * result_bytes(lead.graph);
    for (size_t k = pos.size(); k-- > 0;) {
      out.push_back(queue[pos[k]]);
      pending.erase(queue[pos[k]]);
      queue.erase(queue.begin() + (long)pos[k]);
    }
    std::reverse(out.begin(), out.end());
    return out;
  }

  // A batch failed before it created the workspace it was admitted with.
  void ws_not_created(int32_t graph, WsKind w) {
    GraphInfo &gi = graphs[graph];
    if (!gi.have_ws[w]) return;
    gi.have_ws[w] = false;
    resident -= gi.ws_bytes[w];
  }

  // The batch of `lanes` requests of `kind` on `graph` finished (or failed).
  void release(int32_t graph, int32_t kind, size_t lanes) {
    in_use -= result_units(kind, lanes) * result_bytes(graph);
  }
};

// One batch on a slot. Dev provides:
//   gr_status prepare(size_t result_bytes)  grow the slot's result buffer
//                                           (may free and reallocate it);
//                                           enqueues nothing
//   gr_status enqueue()                     the batch's kernels and result
//                                           copies; may fail after part of
//                                           the work is enqueued
//   gr_status wait_idle()                   wait for all work the slot
//                                           enqueued (bounded; GR_ETIMEOUT)
//   gr_status check_device_errors()         device-side limits of the run
// Whatever happens, a slot never frees, reallocates or reuses a buffer
// while work it enqueued may still run: once enqueue() has been called —
// whether it failed or not — the batch waits for the slot's stream before
// it ends.
template <class Dev>
gr_status run_batch(Dev &dev, size_t result_bytes) {
  gr_status st = dev.prepare(result_bytes);
  if (st != GR_OK) return st;
  st = dev.enqueue();
  const gr_status w = dev.wait_idle();
  if (st == GR_OK) st = w;
  if (st == GR_OK) st = dev.check_device_errors();
  return st;
}

}  // namespace serve
}  // namespace gr
