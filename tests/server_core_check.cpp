// CPU checks of the query server's host-only core (server_core.hpp): the
// batch life cycle against a fake device that records every buffer
// reallocation made while enqueued work may still run, and admission under
// a memory budget. Built and run by tests/test_serving_host.py with g++.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "server_core.hpp"

using namespace gr;
using namespace gr::serve;

static int g_failures = 0;
#define CHECK(cond)                                                    \
  do {                                                                 \
    if (!(cond)) {                                                     \
      std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #cond);       \
      ++g_failures;                                                    \
    }                                                                  \
  } while (0)

// A fake slot: enqueue() leaves work "in flight" (also when it fails after
// enqueueing part of a batch); only wait_idle() retires it. A buffer grown
// while work is in flight is the use-after-free the life cycle must rule out.
struct FakeDev {
  size_t buf_bytes = 0;
  bool in_flight = false;
  int reallocs_in_flight = 0;
  int waits = 0;
  gr_status enqueue_result = GR_OK;
  bool enqueue_touches_device = true;  // failed before any work when false

  gr_status prepare(size_t need) {
    if (buf_bytes < need) {
      if (in_flight) ++reallocs_in_flight;
      buf_bytes = need;
    }
    return GR_OK;
  }
  gr_status enqueue() {
    if (enqueue_touches_device) in_flight = true;
    return enqueue_result;
  }
  gr_status wait_idle() {
    ++waits;
    in_flight = false;
    return GR_OK;
  }
  gr_status check_device_errors() { return GR_OK; }
};

// The order of the earlier worker: it waited for the stream only when every
// step had succeeded. Kept here to show that the fake catches that fault.
static gr_status run_batch_skipping_wait_on_error(FakeDev &d, size_t need) {
  gr_status st = d.prepare(need);
  if (st == GR_OK) st = d.enqueue();
  if (st == GR_OK) st = d.wait_idle();
  return st;
}

static void lifecycle() {
  // a batch whose enqueue fails after enqueueing work, then a larger batch
  {
    FakeDev d;
    d.enqueue_result = GR_ECUDA;
    CHECK(run_batch(d, 1000) == GR_ECUDA);
    CHECK(!d.in_flight);  // the failed batch was waited for
    d.enqueue_result = GR_OK;
    CHECK(run_batch(d, 5000) == GR_OK);  // grows the buffer
    CHECK(d.reallocs_in_flight == 0);
    CHECK(d.waits == 2);
  }
  // the same sequence through the earlier order reallocates under work
  {
    FakeDev d;
    d.enqueue_result = GR_ECUDA;
    run_batch_skipping_wait_on_error(d, 1000);
    d.enqueue_result = GR_OK;
    run_batch_skipping_wait_on_error(d, 5000);
    CHECK(d.reallocs_in_flight == 1);
  }
  // a failure before any device work still ends with the slot idle
  {
    FakeDev d;
    d.enqueue_result = GR_EINVAL;
    d.enqueue_touches_device = false;
    CHECK(run_batch(d, 10) == GR_EINVAL);
    CHECK(!d.in_flight);
  }
}

static Admission make(size_t budget, int32_t max_batch) {
  Admission a;
  a.budget = budget;
  a.max_batch = max_batch;
  return a;
}

static void submit(Admission &a, uint64_t t, int32_t graph, int32_t kind) {
  a.pending[t] = Pending{graph, kind};
  a.queue.push_back(t);
}

static void admission() {
  // graph 0: n = 1000 (4000-byte results), batchable at once; BFS batch
  // workspace 100 kB, single BFS workspace 10 kB
  GraphInfo g0;
  g0.n = 1000;
  g0.min_batch = 1;
  g0.sssp_lanes = 4;
  g0.ws_bytes[kWsBfs] = 10000;
  g0.ws_bytes[kWsBfsBatch] = 100000;
  g0.ws_bytes[kWsSssp] = 20000;
  g0.ws_bytes[kWsSsspBatch] = 80000;
  g0.ws_bytes[kWsCc] = 5000;
  // graph 1: a grid whose BFS requests batch once 3 are queued
  GraphInfo g1 = g0;
  g1.min_batch = 3;

  // plenty of budget: same-graph BFS requests batch in arrival order, other
  // kinds and graphs stay queued in order
  {
    Admission a = make(1 << 20, 64);
    a.graphs = {g0, g1};
    submit(a, 1, 0, GR_QUERY_BFS);
    submit(a, 2, 1, GR_QUERY_BFS);
    submit(a, 3, 0, GR_QUERY_SSSP);
    submit(a, 4, 0, GR_QUERY_BFS);
    submit(a, 5, 0, GR_QUERY_BFS);
    std::vector<uint64_t> b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{1, 4, 5}));
    CHECK(a.in_use == 3 * 4000);
    CHECK(a.resident == 100000);  // the batch workspace was accounted
    a.release(0, GR_QUERY_BFS, b.size());
    CHECK(a.in_use == 0);
    // graph 1 has one BFS request queued, below its batching depth
    b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{2}));
    CHECK(a.resident == 100000 + 10000);
    a.release(1, GR_QUERY_BFS, 1);
    b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{3}));
    a.release(0, GR_QUERY_SSSP, 1);
    CHECK(a.queue.empty() && a.pending.empty());
  }
  // batching depth: three queued BFS requests on graph 1 batch, SSSP lanes
  // stop at the graph's lane limit
  {
    Admission a = make(1 << 20, 64);
    a.graphs = {g0, g1};
    for (uint64_t t = 1; t <= 3; ++t) submit(a, t, 1, GR_QUERY_BFS);
    for (uint64_t t = 4; t <= 10; ++t) submit(a, t, 0, GR_QUERY_SSSP);
    std::vector<uint64_t> b = a.take_batch();
    CHECK(b.size() == 3);
    a.release(1, GR_QUERY_BFS, 3);
    b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{4, 5, 6, 7}));
    a.release(0, GR_QUERY_SSSP, 4);
  }
  // a budget too small for the batch workspace falls back to single
  // requests; the oldest request is admitted alone even when nothing fits
  {
    Admission a = make(50000, 64);
    a.graphs = {g0};
    for (uint64_t t = 1; t <= 5; ++t) submit(a, t, 0, GR_QUERY_BFS);
    std::vector<uint64_t> b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{1}));
    CHECK(a.resident == 10000);
    // while that request is in flight nothing else is admitted if it does
    // not fit: 10000 + 4000 in use + 4000 more still fits here
    a.release(0, GR_QUERY_BFS, 1);
    Admission tiny = make(100, 64);
    tiny.graphs = {g0};
    submit(tiny, 1, 0, GR_QUERY_CC);
    submit(tiny, 2, 0, GR_QUERY_CC);
    b = tiny.take_batch();
    CHECK((b == std::vector<uint64_t>{1}));  // nothing in flight: admitted
    b = tiny.take_batch();
    CHECK(b.empty());  // the first is still in flight and the budget is spent
    tiny.release(0, GR_QUERY_CC, 1);
    b = tiny.take_batch();
    CHECK((b == std::vector<uint64_t>{2}));
  }
  // a workspace that could not be created is no longer counted
  {
    Admission a = make(1 << 20, 1);
    a.graphs = {g0};
    submit(a, 1, 0, GR_QUERY_SSSP);
    std::vector<uint64_t> b = a.take_batch();
    CHECK(a.resident == 20000);
    a.ws_not_created(0, kWsSssp);
    a.release(0, GR_QUERY_SSSP, 1);
    CHECK(a.resident == 0 && a.in_use == 0);
  }
  // the CC requests of a graph share one run: one batch, one result buffer
  {
    Admission a = make(1 << 20, 64);
    a.graphs = {g0, g1};
    submit(a, 1, 0, GR_QUERY_CC);
    submit(a, 2, 1, GR_QUERY_CC);
    submit(a, 3, 0, GR_QUERY_BFS);
    submit(a, 4, 0, GR_QUERY_CC);
    submit(a, 5, 0, GR_QUERY_CC);
    std::vector<uint64_t> b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{1, 4, 5}));
    CHECK(a.in_use == 4000);       // one result, however many requests
    CHECK(a.resident == 5000);     // the CC workspace
    a.release(0, GR_QUERY_CC, b.size());
    CHECK(a.in_use == 0);
    b = a.take_batch();
    CHECK((b == std::vector<uint64_t>{2}));
    a.release(1, GR_QUERY_CC, 1);
  }
  // max_batch = 1 (the plain path) never batches
  {
    Admission a = make(1 << 20, 1);
    a.graphs = {g0};
    for (uint64_t t = 1; t <= 4; ++t) submit(a, t, 0, GR_QUERY_BFS);
    CHECK(a.take_batch().size() == 1);
    Admission c = make(1 << 20, 1);
    c.graphs = {g0};
    for (uint64_t t = 1; t <= 3; ++t) submit(c, t, 0, GR_QUERY_CC);
    CHECK(c.take_batch().size() == 1);
  }
}

int main() {
  lifecycle();
  admission();
  if (g_failures) {
    std::printf("%d failures\n", g_failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
