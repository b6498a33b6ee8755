// Batched form of the C ABI: several independent detection problems
// ("cells") drained by persistent kernels through device ticket counters, the
// tile autotuner, and the CUDA-graph wrapper.  See include/ocd.h.
//
// Planning (host, per call): every non-empty cell is assigned an arrangement
// (residual or bulk-copy projected form) and its tiles -- from the tune table
// when it has an entry for the cell's (B, U, T, storage), else the defaults
// of the single-problem path.  Cells that run the same kernel instance form a
// family; a family is split into launches of at most kBatchCellsPerLaunch
// cells, each launch with its own ticket counter in the workspace and its
// cell table passed by value as the kernel parameter.  The launches go to up
// to four internal streams (heaviest first) so that one family's tail overlaps
// the next family's blocks.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "ocd.h"
#include "ocd_batch.cuh"
#include "ocd_host.h"
#include "ocd_residual.cuh"

using namespace ocdh;

// Ticket counters of ocd_detect_batched_static, the entry point for callers
// that cannot allocate device memory (1 KiB, held by every GPU that loads
// the library): one per launch, and a call makes at most one launch per
// non-empty cell.  Host code must not pass this name to a kernel (it is the
// host-side stand-in); static_scratch() gives the device address.
static __device__ __align__(256) unsigned int g_static_tickets[OCD_STATIC_MAX_CELLS];

namespace {

constexpr int kDefaultStepsPerTicket = 8;  // bulk-copy form: staged steps per ticket

struct CellPlan {
  int index;              // position in the caller's list
  int kind;               // 0 residual, 1 bulk-copy projected, 2 one lane per subcarrier,
                          // 3 tcgen05 projected (a one-cell launch)
  int npp, S, nt, ut;     // kernel instance
  bool fused;             // 32-user kernel with q0 in the G phase (T <= 8)
  size_t smem;
  ocd::DetectParams P;
  long long tickets;
  int sc_per_tick;
  double work;            // rough cost, orders the launches
};

const ocd_tune_entry_t* find_tune(const ocd_tune_t* tune, const ocd_cell_t& c) {
  if (!tune) return nullptr;
  const int n = std::min(std::max(tune->n, 0), OCD_TUNE_MAX_ENTRIES);
  for (int i = 0; i < n; ++i) {
    const ocd_tune_entry_t& e = tune->entry[i];
    if (e.B == c.B && e.U == c.U && e.T == c.T && e.storage == c.storage) return &e;
  }
  return nullptr;
}

// Arrangement and tiles of one cell.  `force` (a tune entry under trial, or
// NULL) overrides the tune table.
int plan_cell(const ocd_cell_t& c, int index, const ocd_tune_t* tune,
              const ocd_tune_entry_t* force, const DeviceInfo& di, CellPlan& cp) {
  Alphabet al;
  int st = validate(c.H, c.Y, c.storage, c.Nsc, c.B, c.U, c.T, c.N0, c.Es, c.K, c.mode,
                    c.qam_order, c.xhat, c.llr, c.algo, al);
  if (st != OCD_OK) return st;
  cp.index = index;
  cp.fused = false;
  build_params(c.H, c.Y, c.storage, c.Nsc, c.B, c.U, c.T, c.N0, c.Es, c.K, c.mode, al, c.xhat,
               c.llr, cp.P);
  const ocd_tune_entry_t* te = force ? force : find_tune(tune, c);
  const bool wide = can_wide(cp.P);
  const bool tma_ok = can_tma32(cp.P) || wide;
  int algo = c.algo;
  // a cell with OCD_ALGO_AUTO takes its shape's tune entry; a tune entry's
  // tcgen05 choice falls back to the default kernel for a cell it does not
  // fit (alignment differs between cells of one shape)
  bool from_tune = false;
  if (algo == OCD_ALGO_AUTO && te && te->algo >= OCD_ALGO_RESIDUAL && te->algo <= OCD_ALGO_PROJECTED_TC) {
    algo = te->algo;
    from_tune = true;
  }
  if (algo == OCD_ALGO_PROJECTED_TC && !can_tc(cp.P)) {
    if (!from_tune)
      return fail(OCD_ERR_UNSUPPORTED, "the tcgen05 kernel needs 16 < U <= 32, T <= %d, float32 "
                  "storage, even B and 16-byte aligned H and Y", ocd::kTcMaxSymbols);
    algo = OCD_ALGO_PROJECTED;
  }
  const bool warp_only = algo == OCD_ALGO_PROJECTED_WARP;
  const bool use_tc = algo == OCD_ALGO_PROJECTED_TC;
  if (warp_only || use_tc) algo = OCD_ALGO_PROJECTED;
  // default without a tune entry: the bulk-copy projected form wherever it
  // applies, one symbol included (as the single-problem path at T = 1)
  if (algo == OCD_ALGO_AUTO) algo = tma_ok ? OCD_ALGO_PROJECTED : OCD_ALGO_RESIDUAL;
  if (algo == OCD_ALGO_PROJECTED && !tma_ok && from_tune) algo = OCD_ALGO_RESIDUAL;
  if (algo == OCD_ALGO_PROJECTED && !tma_ok)
    return fail(OCD_ERR_UNSUPPORTED, "batched projected form needs float32 storage, even B "
                "and 16-byte aligned H and Y (U=%d B=%d)", c.U, c.B);
  if (algo == OCD_ALGO_PROJECTED && can_lane(cp.P)) {
    // one symbol, U <= 8: the single-problem path's one-lane-per-subcarrier
    // kernel, launched for this cell alone (same kernel, same results)
    cp.kind = 2;
    cp.ut = c.U;
    cp.npp = cp.S = 0;
    cp.nt = ocd::projected_lane_threads();
    cp.smem = ocd::projected_lane_smem_per_cta(c.U);
    cp.sc_per_tick = 0;
    cp.tickets = 0;
    cp.work = (double)c.Nsc * (8.0 * c.B * c.U + 8.0 * c.B + 12.0 * c.U);
    return OCD_OK;
  }
  if (algo == OCD_ALGO_PROJECTED && (use_tc || (!warp_only && prefer_tc_batched(cp.P)))) {
    // 17-32 users, 9-16 symbols by default (any T <= 16 when asked for): the
    // single-problem path's tcgen05 kernel,
    // launched for this cell alone (one CTA per SM, same results)
    cp.kind = 3;
    cp.ut = 4;
    cp.npp = cp.S = 0;
    cp.nt = ocd::projected_tc_threads();
    cp.smem = ocd::projected_tc_smem_per_cta(c.T);
    cp.sc_per_tick = 0;
    cp.tickets = 0;
    cp.work = (double)c.Nsc * (8.0 * c.B * c.U + 8.0 * c.T * c.B + 12.0 * c.T * c.U);
    return OCD_OK;
  }
  if (algo == OCD_ALGO_PROJECTED) {
    cp.kind = 1;
    cp.ut = c.U <= 8 ? 1 : c.U <= 16 ? 2 : 4;
    cp.fused = wide && ocd::wide_fuses(c.T);
    cp.npp = cp.S = 0;
    cp.nt = wide ? ocd::projected_wide_threads() : ocd::projected_tma_threads();
    cp.smem = wide ? ocd::projected_wide_smem_per_cta() : ocd::projected_tma_smem_per_cta(c.U);
    int spt = te && te->sc_per_ticket > 0 ? te->sc_per_ticket : 0;
    if (spt == 0) {
      const int steps = ocd::tma_steps_per_sc(c.B, c.T) + (wide ? (c.B + 31) / 32 : 0);
      spt = (kDefaultStepsPerTicket + steps - 1) / steps;
    }
    if (spt < 1 || spt > 256) return fail(OCD_ERR_ARG, "sc_per_ticket=%d outside 1..256", spt);
    cp.sc_per_tick = spt;
    cp.tickets = (c.Nsc + spt - 1) / spt;
    cp.work = (double)c.Nsc * (8.0 * c.B * c.U + 8.0 * c.T * c.B + 12.0 * c.T * c.U);
    return OCD_OK;
  }
  cp.kind = 0;
  cp.ut = 0;
  int S_req = te ? te->symbols_per_item : 0;
  int L_req = te ? te->lanes_per_item : 0;
  if (S_req < 0 || S_req > 2) return fail(OCD_ERR_ARG, "symbols_per_item=%d outside 0..2", S_req);
  if (L_req < 0 || L_req > 32 || (L_req & (L_req - 1)))
    return fail(OCD_ERR_ARG, "lanes_per_item=%d is not a power of two <= 32", L_req);
  if (c.T < 2) S_req = 1;
  Plan pl;
  st = make_plan(c.B, c.U, c.T, kSmemBudget, cp.P, pl, S_req, L_req);
  if (st != OCD_OK)
    st = make_plan(c.B, c.U, c.T, di.smem_optin - kBatchStaticSmem, cp.P, pl, S_req, L_req);
  if (st != OCD_OK) return st;
  cp.npp = pl.npp;
  cp.S = pl.S;
  cp.nt = pl.nt;
  cp.smem = pl.smem;
  cp.sc_per_tick = 0;
  cp.tickets = (cp.P.items + cp.P.chunk - 1) / cp.P.chunk;
  cp.work = (double)c.Nsc * c.T * (8.0 * c.B * c.U * (c.K + 0.25));
  return OCD_OK;
}

bool same_family(const CellPlan& a, const CellPlan& b) {
  return a.kind == b.kind && a.npp == b.npp && a.S == b.S && a.nt == b.nt && a.ut == b.ut &&
         a.fused == b.fused;
}

struct Launch {
  const void* fn;
  unsigned grid;
  int nt;
  size_t smem;
  double work;
  std::unique_ptr<ocd::BatchTable> tab;  // persistent launches: the cell table
  bool single = false;                   // one-cell launch with parameters P
  ocd::DetectParams P;
  std::unique_ptr<CUtensorMap> map;      // one-cell tcgen05 launch: its tensor map
};

// Plans every cell and groups them into launches (heaviest first).
int plan_batch(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
               const ocd_tune_entry_t* force, const DeviceInfo& di,
               std::vector<Launch>& launches) {
  std::vector<CellPlan> plans;
  plans.reserve(ncells);
  for (int i = 0; i < ncells; ++i) {
    const ocd_cell_t& c = cells[i];
    CellPlan cp;
    const int st = plan_cell(c, i, tune, force, di, cp);
    if (st != OCD_OK) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", ocd_last_error());
      return fail(st, "cell %d: %s", i, msg);
    }
    if ((long long)c.Nsc * c.T == 0) continue;
    plans.push_back(cp);
  }
  // families in order of first appearance; each split into launches
  std::vector<bool> taken(plans.size(), false);
  for (size_t i = 0; i < plans.size(); ++i) {
    if (taken[i]) continue;
    if (plans[i].kind == 2) {
      taken[i] = true;
      Launch L;
      L.single = true;
      L.P = plans[i].P;
      L.fn = ocd::projected_lane_kernel_ptr(plans[i].P.U);
      L.nt = plans[i].nt;
      L.smem = plans[i].smem;
      L.work = plans[i].work;
      const int st = lane_grid(L.P, di, L.grid);
      if (st != OCD_OK) return st;
      if (L.grid == 0)
        return fail(OCD_ERR_UNSUPPORTED, "cell %d: one-lane kernel cannot be resident", plans[i].index);
      launches.push_back(std::move(L));
      continue;
    }
    if (plans[i].kind == 3) {
      taken[i] = true;
      Launch L;
      L.single = true;
      L.P = plans[i].P;
      L.fn = ocd::projected_tc_kernel_ptr(plans[i].P.T);
      L.nt = plans[i].nt;
      L.smem = plans[i].smem;
      L.work = plans[i].work;
      L.map.reset(new CUtensorMap);
      const cudaError_t e = ocd::encode_ymap_rows(L.P, L.map.get(), L.P.T <= 8 ? 8 : 16);
      if (e == cudaErrorNotSupported)
        return fail(OCD_ERR_UNSUPPORTED, "cell %d: no tensor-map encoder in this driver", plans[i].index);
      if (e != cudaSuccess) return fail(OCD_ERR_CUDA, "cell %d: tensor map encoding failed", plans[i].index);
      L.grid = (unsigned)std::min<long long>(di.sms, L.P.Nsc);  // one CTA per SM, persistent
      launches.push_back(std::move(L));
      continue;
    }
    std::vector<size_t> fam;
    for (size_t j = i; j < plans.size(); ++j)
      if (!taken[j] && same_family(plans[i], plans[j])) {
        fam.push_back(j);
        taken[j] = true;
      }
    for (size_t a = 0; a < fam.size(); a += ocd::kBatchCellsPerLaunch) {
      const size_t b = std::min(fam.size(), a + (size_t)ocd::kBatchCellsPerLaunch);
      Launch L;
      L.tab.reset(new ocd::BatchTable);
      memset(L.tab.get(), 0, sizeof(ocd::BatchTable));
      const CellPlan& f = plans[fam[a]];
      L.fn = f.kind == 0 ? reinterpret_cast<const void*>(ocd::batched_residual_kernel(f.npp, f.S))
             : f.ut == 4 ? reinterpret_cast<const void*>(ocd::batched_wide_kernel(f.fused))
                         : reinterpret_cast<const void*>(ocd::batched_tma_kernel(f.ut == 1 ? 8 : 16));
      L.nt = f.nt;
      L.smem = 0;
      L.work = 0.0;
      long long tick = 0;
      for (size_t k = a; k < b; ++k) {
        const CellPlan& cp = plans[fam[k]];
        ocd::BatchCell& bc = L.tab->cell[k - a];
        bc.P = cp.P;
        if (cp.kind == 1) {
          // the 8/16-user bulk-copy kernel takes the 3-D view where B allows;
          // the 32-user kernel copies 16-antenna boxes (2-D view)
          const cudaError_t e = cp.ut == 4 ? ocd::encode_ymap(cp.P, &bc.ymap)
                                           : ocd::encode_ymap_tma(cp.P, &bc.ymap, &bc.P.ymap3d);
          if (e == cudaErrorNotSupported)
            return fail(OCD_ERR_UNSUPPORTED, "cell %d: no tensor-map encoder in this driver", cp.index);
          if (e != cudaSuccess) return fail(OCD_ERR_CUDA, "cell %d: tensor map encoding failed", cp.index);
        }
        tick += cp.tickets;
        bc.tick_end = tick;
        bc.sc_per_tick = cp.sc_per_tick;
        L.smem = std::max(L.smem, cp.smem);
        L.work += cp.work;
      }
      if (tick >= 0xffffffffll) return fail(OCD_ERR_UNSUPPORTED, "too many tickets in one launch");
      L.tab->total = (unsigned int)tick;
      L.tab->ncells = (int)(b - a);
      int per_sm = 0;
      const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L.fn, L.nt, L.smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (per_sm < 1) return fail(OCD_ERR_UNSUPPORTED, "batched kernel cannot be resident (smem %zu)", L.smem);
      long long grid = (long long)di.sms * per_sm;
      const long long units = f.kind == 1 ? (tick + L.nt / 32 - 1) / (L.nt / 32) : tick;
      if (grid > units) grid = units;
      L.grid = (unsigned)grid;
      launches.push_back(std::move(L));
    }
  }
  std::stable_sort(launches.begin(), launches.end(),
                   [](const Launch& x, const Launch& y) { return x.work > y.work; });
  return OCD_OK;
}

// Every cell's arguments, before any CUDA call.
int check_cells(const ocd_cell_t* cells, int ncells) {
  if (ncells < 0 || ncells > OCD_MAX_CELLS)
    return fail(OCD_ERR_ARG, "ncells=%d outside 0..%d", ncells, OCD_MAX_CELLS);
  if (ncells > 0 && !cells) return fail(OCD_ERR_ARG, "cells must not be NULL");
  for (int i = 0; i < ncells; ++i) {
    const ocd_cell_t& c = cells[i];
    Alphabet al;
    const int st = validate(c.H, c.Y, c.storage, c.Nsc, c.B, c.U, c.T, c.N0, c.Es, c.K, c.mode,
                            c.qam_order, c.xhat, c.llr, c.algo, al);
    if (st != OCD_OK) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", ocd_last_error());
      return fail(st, "cell %d: %s", i, msg);
    }
  }
  return OCD_OK;
}

int check_batch_args(const ocd_cell_t* cells, int ncells, void* workspace, size_t bytes) {
  if (ncells < 0 || ncells > OCD_MAX_CELLS)
    return fail(OCD_ERR_ARG, "ncells=%d outside 0..%d", ncells, OCD_MAX_CELLS);
  if (ncells > 0 && !cells) return fail(OCD_ERR_ARG, "cells must not be NULL");
  if (ncells > 0 && (!workspace || ((uintptr_t)workspace & 3u)))
    return fail(OCD_ERR_ARG, "workspace must be a 4-byte aligned device pointer");
  if (ncells > 0 && bytes < ocd_batched_workspace_size(ncells))
    return fail(OCD_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed", bytes,
                ocd_batched_workspace_size(ncells));
  return check_cells(cells, ncells);
}

// Enqueues the planned launches: counters zeroed on `stream`, then the
// launches on the internal streams (or on `stream` when there is one).
int enqueue(std::vector<Launch>& launches, void* workspace, cudaStream_t stream) {
  if (launches.empty()) return OCD_OK;
  unsigned int* counters = static_cast<unsigned int*>(workspace);
  cudaError_t e = cudaMemsetAsync(counters, 0, launches.size() * sizeof(unsigned int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  // a persistent launch takes (cell table, its ticket counter); a one-cell
  // launch takes the cell's parameters
  auto launch = [&](Launch& L, unsigned int* ctr, cudaStream_t s) {
    if (L.single && L.map) {
      void* args[] = {&L.P, L.map.get()};
      return cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.nt), args, L.smem, s);
    }
    if (L.single) {
      void* args[] = {&L.P};
      return cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.nt), args, L.smem, s);
    }
    void* args[] = {L.tab.get(), &ctr};
    return cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.nt), args, L.smem, s);
  };
  if (launches.size() == 1) {
    e = launch(launches[0], counters, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
    return OCD_OK;
  }
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_hs_mu);
  HostStreams* hs = nullptr;
  int st = host_streams(dev, hs);
  if (st != OCD_OK) return st;
  const int ns = (int)std::min(launches.size(), (size_t)kHostStreams);
  e = cudaEventRecord(hs->ev_in, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  for (int i = 0; i < ns; ++i) {
    e = cudaStreamWaitEvent(hs->s[i], hs->ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  for (size_t i = 0; i < launches.size(); ++i) {
    e = launch(launches[i], counters + i, hs->s[i % ns]);
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
  }
  for (int i = 0; i < ns; ++i) {
    e = cudaEventRecord(hs->ev_out[i], hs->s[i]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    e = cudaStreamWaitEvent(stream, hs->ev_out[i], 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  return OCD_OK;
}

int run_batch(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
              const ocd_tune_entry_t* force, void* workspace, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceInfo di;
  int st = device_info(dev, di);
  if (st != OCD_OK) return st;
  std::vector<Launch> launches;
  st = plan_batch(cells, ncells, tune, force, di, launches);
  if (st != OCD_OK) return st;
  st = enqueue(launches, workspace, stream);
  if (st == OCD_OK) {
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  }
  return st;
}

struct StaticScratch {
  bool ready = false;
  unsigned int* ptr = nullptr;
};
StaticScratch g_static[kMaxDevices];
std::mutex g_static_mu;

// Device address of g_static_tickets on `dev` (the current device), looked
// up once per device.  The same first call also creates the device's
// internal streams and events (what an enqueue of several kernel families
// uses), so that no later call creates them, whether or not that later call
// runs under a stream capture.
int static_scratch(int dev, unsigned int*& out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(OCD_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static[dev].ready) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_tickets);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    {
      std::lock_guard<std::mutex> lk_hs(g_hs_mu);  // lock order: g_static_mu, then g_hs_mu
      HostStreams* hs = nullptr;
      const int st = host_streams(dev, hs);
      if (st != OCD_OK) return st;
    }
    g_static[dev].ptr = static_cast<unsigned int*>(p);
    g_static[dev].ready = true;
  }
  out = g_static[dev].ptr;
  return OCD_OK;
}

}  // namespace

struct ocd_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

extern "C" {

size_t ocd_batched_workspace_size(int ncells) {
  if (ncells <= 0) return 0;
  const size_t b = (size_t)ncells * sizeof(unsigned int);
  return (b + 255) / 256 * 256;
}

int ocd_detect_batched(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                       void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  int st = check_batch_args(cells, ncells, workspace, workspace_bytes);
  if (st != OCD_OK || ncells == 0) return st;
  return run_batch(cells, ncells, tune, nullptr, workspace, stream);
}

int ocd_detect_batched_static(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                              cudaStream_t stream) {
  if (ncells > OCD_STATIC_MAX_CELLS)
    return fail(OCD_ERR_UNSUPPORTED, "ncells=%d exceeds the %d cells of the static scratch", ncells,
                OCD_STATIC_MAX_CELLS);
  int st = check_cells(cells, ncells);
  if (st != OCD_OK || ncells == 0) return st;
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  unsigned int* tickets = nullptr;
  st = static_scratch(dev, tickets);
  if (st != OCD_OK) return st;
  return run_batch(cells, ncells, tune, nullptr, tickets, stream);
}

int ocd_autotune_batched(const ocd_cell_t* cells, int ncells, void* workspace,
                         size_t workspace_bytes, int reps, ocd_tune_t* tune,
                         cudaStream_t stream) {
  int st = check_batch_args(cells, ncells, workspace, workspace_bytes);
  if (st != OCD_OK) return st;
  if (!tune) return fail(OCD_ERR_ARG, "tune must not be NULL");
  if (reps < 1 || reps > 100) return fail(OCD_ERR_ARG, "reps=%d outside 1..100", reps);
  // validate everything first, so that a bad cell enqueues nothing
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    DeviceInfo di;
    st = device_info(dev, di);
    if (st != OCD_OK) return st;
    std::vector<Launch> probe;
    st = plan_batch(cells, ncells, nullptr, nullptr, di, probe);
    if (st != OCD_OK) return st;
  }
  ocd_tune_t out;
  memset(&out, 0, sizeof(out));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  // Mean time (us) of `reps` enqueues of `n` cells after one warm-up, with
  // the tune table `t` or the single entry `force`.
  auto time_run = [&](const ocd_cell_t* cs, int n, const ocd_tune_t* t,
                      const ocd_tune_entry_t* force, float& us) -> int {
    int s2 = run_batch(cs, n, t, force, workspace, stream);  // warm-up
    if (s2 != OCD_OK) return s2;
    cudaError_t ee = cudaEventRecord(e0, stream);
    for (int r = 0; r < reps && s2 == OCD_OK && ee == cudaSuccess; ++r)
      s2 = run_batch(cs, n, t, force, workspace, stream);
    if (ee == cudaSuccess) ee = cudaEventRecord(e1, stream);
    if (ee == cudaSuccess) ee = cudaEventSynchronize(e1);
    if (s2 != OCD_OK) return s2;
    if (ee != cudaSuccess) return cuda_fail(ee, "autotune timing");
    float ms = 0.0f;
    ee = cudaEventElapsedTime(&ms, e0, e1);
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaEventElapsedTime");
    us = 1000.0f * ms / reps;
    return OCD_OK;
  };

  // Phase 1: per shape, the fastest tile on that shape's cells alone.
  struct Shape {
    std::vector<ocd_cell_t> group;  // the shape's cells (algo AUTO)
    bool tma_all = false;           // every cell takes the projected form
    bool lane_all = false;          // every cell runs the one-lane kernel
    bool tc_all = false;            // every cell fits the tcgen05 kernel
    bool wide = false;              // 17-32 users
  };
  std::vector<Shape> shapes;
  std::vector<bool> done(ncells, false);
  for (int i = 0; i < ncells && st == OCD_OK; ++i) {
    const ocd_cell_t& c = cells[i];
    if (done[i] || (long long)c.Nsc * c.T == 0) continue;
    Shape sh;
    for (int j = i; j < ncells; ++j) {
      const ocd_cell_t& d = cells[j];
      if (!done[j] && d.B == c.B && d.U == c.U && d.T == c.T && d.storage == c.storage &&
          (long long)d.Nsc * d.T > 0) {
        ocd_cell_t g = d;
        g.algo = OCD_ALGO_AUTO;  // the candidate decides
        sh.group.push_back(g);
        done[j] = true;
      }
    }
    if (out.n >= OCD_TUNE_MAX_ENTRIES) {
      st = fail(OCD_ERR_UNSUPPORTED, "more than %d distinct shapes", OCD_TUNE_MAX_ENTRIES);
      break;
    }
    // candidates: projected (if the shape takes it) x tickets; residual x S x L
    std::vector<ocd_tune_entry_t> cand;
    Alphabet al;
    alphabet_of(c.qam_order, al);
    const ocd_tune_entry_t base = {c.B, c.U, c.T, c.storage, 0, 0, 0, 0, 0.0f};
    sh.tma_all = sh.lane_all = sh.tc_all = true;
    sh.wide = c.U > 16;
    for (const ocd_cell_t& g : sh.group) {
      ocd::DetectParams Pg;
      build_params(g.H, g.Y, g.storage, g.Nsc, g.B, g.U, g.T, g.N0, g.Es, g.K, g.mode, al,
                   g.xhat, g.llr, Pg);
      sh.tma_all = sh.tma_all && (can_tma32(Pg) || can_wide(Pg));
      sh.lane_all = sh.lane_all && can_lane(Pg);
      sh.tc_all = sh.tc_all && can_tc(Pg);
    }
    if (sh.lane_all) {  // the one-lane kernel has no tile to choose
      ocd_tune_entry_t t = base;
      t.algo = OCD_ALGO_PROJECTED;
      cand.push_back(t);
    } else if (sh.tma_all && c.T >= 1) {
      for (int spt : {1, 2, 4, 8, 16, 32}) {
        ocd_tune_entry_t t = base;
        t.algo = OCD_ALGO_PROJECTED;
        t.sc_per_ticket = spt;
        cand.push_back(t);
      }
    }
    for (int S = 1; S <= (c.T >= 2 ? 2 : 1); ++S) {
      int L0 = 1;
      while (L0 * 8 < (c.B + 1) / 2) L0 <<= 1;
      for (int L = L0; L <= 32 && L <= 4 * L0; L <<= 1) {
        ocd_tune_entry_t t = base;
        t.algo = OCD_ALGO_RESIDUAL;
        t.symbols_per_item = S;
        t.lanes_per_item = L;
        cand.push_back(t);
      }
    }
    float best = INFINITY;
    ocd_tune_entry_t pick = base;
    for (const ocd_tune_entry_t& t : cand) {
      float us = 0.0f;
      const int s2 = time_run(sh.group.data(), (int)sh.group.size(), nullptr, &t, us);
      if (s2 == OCD_ERR_UNSUPPORTED) continue;  // e.g. the tile does not fit
      if (s2 != OCD_OK) { st = s2; break; }
      if (us < best) {
        best = us;
        pick = t;
        pick.time_us = us;
      }
    }
    if (st == OCD_OK) {
      if (!(best < INFINITY)) st = fail(OCD_ERR_UNSUPPORTED, "no tile fits shape B=%d U=%d T=%d", c.B, c.U, c.T);
      else {
        out.entry[out.n++] = pick;
        shapes.push_back(std::move(sh));
      }
    }
  }

  // Phase 2: the whole batch.  Shapes timed alone do not show how their
  // launches share the GPU on the internal streams (a tcgen05 launch holds
  // every SM it runs on; persistent launches of other kernels fill SMs as
  // they free up), so the table is refined on all cells at once: the
  // defaults as a whole, then one shape at a time its other choices
  // (kernel of a 32-user shape, tickets halved or doubled, the other
  // arrangement), each kept only when the whole batch gets faster by more
  // than the noise margin.
  if (st == OCD_OK && out.n > 0) {
    constexpr float kKeep = 0.985f;  // a change must save more than 1.5%
    float best = 0.0f;
    st = time_run(cells, ncells, &out, nullptr, best);
    // the defaults, written out as explicit entries (tiles left at zero)
    ocd_tune_t def = out;
    for (int i = 0; i < def.n; ++i) {
      ocd_tune_entry_t& t = def.entry[i];
      t.algo = shapes[i].tma_all ? OCD_ALGO_PROJECTED : OCD_ALGO_RESIDUAL;
      t.symbols_per_item = t.lanes_per_item = t.sc_per_ticket = 0;
      t.time_us = 0.0f;
    }
    float us = 0.0f;
    if (st == OCD_OK) st = time_run(cells, ncells, &def, nullptr, us);
    if (st == OCD_OK && us < kKeep * best) {
      out = def;
      best = us;
    }
    // one kernel for every 17-32-user shape at once (their launches share
    // the SMs with each other, so single changes can each stay under the
    // margin while the joint one does not)
    for (int a : {OCD_ALGO_PROJECTED_WARP, OCD_ALGO_PROJECTED_TC}) {
      if (st != OCD_OK) break;
      ocd_tune_t trial = out;
      int changed = 0;
      for (int i = 0; i < trial.n; ++i) {
        ocd_tune_entry_t& t = trial.entry[i];
        const bool proj = t.algo == OCD_ALGO_PROJECTED || t.algo == OCD_ALGO_PROJECTED_WARP ||
                          t.algo == OCD_ALGO_PROJECTED_TC;
        if (shapes[i].wide && shapes[i].tc_all && proj && t.algo != a) {
          t.algo = a;
          t.time_us = 0.0f;
          ++changed;
        }
      }
      if (changed < 2) continue;  // a single shape is tried below
      const int s2 = time_run(cells, ncells, &trial, nullptr, us);
      if (s2 == OCD_ERR_UNSUPPORTED) continue;
      if (s2 != OCD_OK) { st = s2; break; }
      if (us < kKeep * best) {
        out = trial;
        best = us;
      }
    }
    for (int i = 0; i < out.n && st == OCD_OK; ++i) {
      const Shape& sh = shapes[i];
      if (sh.lane_all) continue;
      std::vector<ocd_tune_entry_t> alt;
      const ocd_tune_entry_t cur = out.entry[i];
      const bool proj = cur.algo == OCD_ALGO_PROJECTED || cur.algo == OCD_ALGO_PROJECTED_WARP ||
                        cur.algo == OCD_ALGO_PROJECTED_TC;
      if (proj) {
        if (sh.wide && sh.tc_all) {
          for (int a : {OCD_ALGO_PROJECTED_WARP, OCD_ALGO_PROJECTED_TC}) {
            ocd_tune_entry_t t = cur;
            t.algo = a;
            if (a != cur.algo) alt.push_back(t);
          }
        }
        const int spt = cur.sc_per_ticket;
        for (int f : {2, -2}) {
          ocd_tune_entry_t t = cur;
          t.sc_per_ticket = spt == 0 ? (f > 0 ? 16 : 1) : (f > 0 ? spt * 2 : spt / 2);
          if (t.sc_per_ticket >= 1 && t.sc_per_ticket <= 256 && t.sc_per_ticket != spt) alt.push_back(t);
        }
        ocd_tune_entry_t r = cur;
        r.algo = OCD_ALGO_RESIDUAL;
        r.symbols_per_item = r.lanes_per_item = r.sc_per_ticket = 0;
        alt.push_back(r);
      } else if (sh.tma_all) {
        ocd_tune_entry_t t = cur;
        t.algo = OCD_ALGO_PROJECTED;
        t.symbols_per_item = t.lanes_per_item = t.sc_per_ticket = 0;
        alt.push_back(t);
      }
      for (const ocd_tune_entry_t& t : alt) {
        ocd_tune_t trial = out;
        trial.entry[i] = t;
        trial.entry[i].time_us = 0.0f;
        const int s2 = time_run(cells, ncells, &trial, nullptr, us);
        if (s2 == OCD_ERR_UNSUPPORTED) continue;
        if (s2 != OCD_OK) { st = s2; break; }
        if (us < kKeep * best) {
          out = trial;
          best = us;
        }
      }
    }
    // entries changed in phase 2 carry the time of their shape alone
    for (int i = 0; i < out.n && st == OCD_OK; ++i) {
      if (out.entry[i].time_us > 0.0f) continue;
      ocd_tune_entry_t t = out.entry[i];
      st = time_run(shapes[i].group.data(), (int)shapes[i].group.size(), nullptr, &t, us);
      if (st == OCD_OK) out.entry[i].time_us = us;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == OCD_OK) *tune = out;
  return st;
}

int ocd_graph_create_batched(const ocd_cell_t* cells, int ncells, const ocd_tune_t* tune,
                             void* workspace, size_t workspace_bytes, ocd_graph_t** graph) {
  if (!graph) return fail(OCD_ERR_ARG, "graph must not be NULL");
  *graph = nullptr;
  int st = check_batch_args(cells, ncells, workspace, workspace_bytes);
  if (st != OCD_OK) return st;
  std::unique_ptr<ocd_graph> g(new ocd_graph);
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // per-device state (kernel attributes, internal streams) exists before
  // the capture starts
  {
    DeviceInfo di;
    st = device_info(g->device, di);
    if (st != OCD_OK) return st;
    std::lock_guard<std::mutex> lk(g_hs_mu);
    HostStreams* hs = nullptr;
    st = host_streams(g->device, hs);
    if (st != OCD_OK) return st;
  }
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  st = ncells > 0 ? run_batch(cells, ncells, tune, nullptr, workspace, cs) : OCD_OK;
  cudaGraph_t cg = nullptr;
  e = cudaStreamEndCapture(cs, &cg);
  cudaStreamDestroy(cs);
  if (st != OCD_OK) {
    if (cg) cudaGraphDestroy(cg);
    return st;
  }
  if (e != cudaSuccess) {
    if (cg) cudaGraphDestroy(cg);
    return cuda_fail(e, "cudaStreamEndCapture");
  }
  g->graph = cg;
  e = cudaGraphInstantiate(&g->exec, cg, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(cg);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  *graph = g.release();
  return OCD_OK;
}

int ocd_graph_launch(ocd_graph_t* graph, cudaStream_t stream) {
  if (!graph || !graph->exec) return fail(OCD_ERR_ARG, "graph must not be NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != graph->device)
    return fail(OCD_ERR_ARG, "graph was created on device %d, current device is %d", graph->device, dev);
  e = cudaGraphLaunch(graph->exec, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return OCD_OK;
}

int ocd_graph_destroy(ocd_graph_t* graph) {
  if (!graph) return OCD_OK;
  cudaError_t e = cudaSuccess;
  if (graph->exec) e = cudaGraphExecDestroy(graph->exec);
  if (graph->graph) {
    const cudaError_t e2 = cudaGraphDestroy(graph->graph);
    if (e == cudaSuccess) e = e2;
  }
  delete graph;
  if (e != cudaSuccess) return cuda_fail(e, "destroying the graph");
  return OCD_OK;
}

}  // extern "C"
