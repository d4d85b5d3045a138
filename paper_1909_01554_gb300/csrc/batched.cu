// Batched products of uneven sizes in one persistent launch, with the base
// case and the tile form of every problem chosen per shape.
//
// A plan is built once on the host. For every problem it decides, from a cost
// model measured on the device (below):
//   - the base-case path: the tensor cores (the plan's tensor path) or the
//     CUDA cores (LOP3/POPC), whichever the model says is faster for the
//     shape (small k and narrow tiles pay more tensor-path padding);
//   - the tile form of its last column tile: N = 128 MMAs where at most 128
//     of its 256 columns lie inside n and the measured N = 128 stage is
//     cheaper than the N = 256 one;
//   - k in operand stages (256 bits e2m1, 128 bits e4m3); an odd count ends
//     in half a packed stage, whose second operand stage is not multiplied;
//   - for a binary product, the Strassen depth a single product of its shape
//     gets (Sec. 3.8); one with depth > 0 runs as its own Strassen product
//     after the batched launches, in plan-held scratch.
// Then it builds per-problem TMA maps over A (or a copy of A with an even row
// pitch) and over the transposed B, the work list of all tensor tiles
// (256 x 256 on SM pairs, 128 x 256 where pairs are unavailable) assigned
// longest-first to the least loaded CTA pair (model cost of each tile), and
// the list of CUDA-core tiles (128 x 128), longest first.
//
// Running a plan only launches kernels: one batched bit transpose of every B,
// one pass that pads rows whose k/64 word count is odd (tensor problems), one
// persistent tensor-core launch over the tensor tiles and, when some problem
// chose the CUDA cores, one persistent CUDA-core launch over theirs, then
// the Strassen problems' own launches. Nothing in a run allocates or
// synchronises, so a run can be captured in a CUDA graph and replayed.
//
// The cost model (per device and tensor path, measured once on the first
// plan that needs it; Sec. 3.17 fixes what memory forces and chooses the
// rest by measurement): synthetic batches of equal problems are timed on
// this device, the tensor kernel at two k (k stages and a fixed cost per
// tile) and with N = 128 tiles, the CUDA-core kernel at two k. A tile's time
// is then stages x (cost per stage) + (cost per tile), divided by the units
// that run tiles side by side.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <queue>
#include <vector>

#include "plan.h"
#include "tc_batched.h"

namespace bmm {

namespace {

// Rows of odd-k tensor problems: copy A rows into the even-pitch buffer
// (zeroing the pad word) and zero the pad word of every Bt row. The work of
// a job is cut into warp items: ga rows of A at a time (ga = 32 / kp rows, so
// short rows still keep every lane busy; one row when it has more than 16
// words), then 32 Bt rows at a time, one lane per row.
struct PadJob {
    const uint64_t* A;
    uint64_t* Apad;
    uint64_t* Bt;
    int64_t m, n, kw, kp;  // kw = k/64 (odd), kp = kw + 1
    int64_t ga, a_items;   // A rows per warp item, warp items of A
};

__global__ void __launch_bounds__(256) pad_kernel(const PadJob* __restrict__ jobs,
                                                  const int64_t* __restrict__ first, int count,
                                                  int64_t total_items) {
    const int lane = threadIdx.x & 31;
    for (int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; it < total_items;
         it += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const PadJob j = jobs[lo];
        const int64_t local = it - first[lo];
        if (local < j.a_items) {
            const int64_t r0 = local * j.ga;
            if (j.ga > 1) {
                const int64_t row = r0 + lane / j.kp, w = lane % j.kp;
                if (lane < j.ga * j.kp && row < j.m)
                    j.Apad[row * j.kp + w] = w < j.kw ? j.A[row * j.kw + w] : 0ull;
            } else {
                for (int64_t w = lane; w < j.kp; w += 32)
                    j.Apad[r0 * j.kp + w] = w < j.kw ? j.A[r0 * j.kw + w] : 0ull;
            }
        } else {
            const int64_t row = (local - j.a_items) * 32 + lane;
            if (row < j.n) j.Bt[row * j.kp + j.kw] = 0ull;
        }
    }
}

uint64_t round256(uint64_t x) { return (x + 255) / 256 * 256; }

// The batched schedule's cost model for one tensor path on one device
// (nanoseconds on one unit: a CTA pair, or a CTA, of each launch).
struct Model {
    bool measured = false;
    int tc_units = 0;           // tensor tiles running side by side
    double tc_stage = 0.0;      // per operand stage of an N = 256 tile
    double tc_stage128 = 0.0;   // per operand stage of an N = 128 tile
    double tc_tile = 0.0;       // per tile: accumulator hand-off, epilogue, start
    int pc_units = 0;           // CUDA-core tiles running side by side
    double pc_stage = 0.0;      // per 256-bit stage of k of a 128 x 128 tile
    double pc_tile = 0.0;       // per tile: epilogue, start
};

// Before measurement: figures of this kernel on a GB300 at ~2 GHz (e2m1 pair
// stage ~650 cycles with the producers' traffic, hand-off ~900 cycles; e4m3
// operand stages carry half the k at about the same time; LOP3 tile stage
// ~1300 cycles). Only used where the device cannot be measured.
Model default_model(int tc_path) {
    Model M;
    M.tc_units = tc_path == BMM_PATH_POPC ? 0
                 : tc_path == BMM_PATH_TC_FP8 ? sm_count()
                                              : std::max(1, sm_count() / 2);
    M.tc_stage = 320.0;
    M.tc_stage128 = 250.0;
    M.tc_tile = 450.0;
    M.pc_units = popc_batched_grid();
    M.pc_stage = 660.0;
    M.pc_tile = 1000.0;
    return M;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// k bits per operand stage of a tensor path.
int64_t op_stage_bits(int path) { return path == BMM_PATH_TC_FP4_PAIR ? 256 : 128; }

}  // namespace
}  // namespace bmm

using namespace bmm;

// What the plan decided for one problem.
struct BatchChoice {
    int path = BMM_PATH_POPC;  // resolved base case
    int n128 = 0;              // tensor: the last column tile runs N = 128 MMAs
    int64_t nks = 0;           // tensor: operand stages of k; CUDA cores: 256-bit stages
    double cost_ns = 0.0;      // model time of all its tiles on one unit
    bool strassen = false;     // runs as its own Strassen product (plan below)
    Plan sp;                   // that product's plan (depth > 0)
};

struct bmm_batched_plan_s {
    int device = 0;
    int count = 0;
    int tc_path = BMM_PATH_POPC;  // the tensor path of the plan's tensor problems
    bool pair = false;            // SM pairs: 256-row tiles, one work list per CTA pair
    bool fp4 = false;             // e2m1 operands (SM pairs only)
    // problem list (host)
    std::vector<int> op;
    std::vector<const uint64_t*> A, B;
    std::vector<uint64_t*> C;
    std::vector<int64_t> m, k, n;
    std::vector<BatchChoice> choice;
    Model model;
    // device memory owned by the plan (one allocation)
    void* dmem = nullptr;
    TcProblem* d_probs = nullptr;
    TcWorkItem* d_items = nullptr;
    int32_t* d_cta_ptr = nullptr;
    TransposeJob* d_tjobs = nullptr;  // load/store-form transposes
    int64_t* d_tfirst = nullptr;
    TmaTransposeJob* d_ttjobs = nullptr;  // TMA-form transposes
    int64_t* d_ttfirst = nullptr;
    int transpose_count = 0, tma_count = 0;
    int64_t tma_total = 0;
    PadJob* d_pjobs = nullptr;
    int64_t* d_pfirst = nullptr;
    PopcJob* d_pcjobs = nullptr;
    PopcTile* d_pctiles = nullptr;
    void* strassen_ws = nullptr;  // inside dmem: scratch of the largest Strassen problem
    int strassen_problems = 0;
    int grid = 0;                 // tensor launch units (0: no tensor problem)
    int64_t pc_tiles = 0;         // CUDA-core tiles (0: no CUDA-core problem)
    int64_t transpose_total = 0, pad_total = 0;
    int pad_count = 0;
    std::vector<uint64_t*> Bt;  // per problem, inside dmem
    std::vector<int64_t> kp;
    // statistics
    int tc_problems = 0, pc_problems = 0;
    int64_t tc_tiles = 0, tc_tiles128 = 0;
    double macs_needed = 0.0, macs_issued = 0.0, est_ms = 0.0;
};

namespace {

// Fills P->choice: req[i] is AUTO (the model decides), BMM_PATH_POPC or the
// plan's tensor path. Tensor-path tails take N = 128 where the model's N =
// 128 stage is the cheaper one.
void decide(bmm_batched_plan_s* P, const int32_t* req) {
    const Model& M = P->model;
    const bool tc = P->tc_path != BMM_PATH_POPC;
    const int64_t kst = tc ? op_stage_bits(P->tc_path) : 256;
    const int64_t tile_m = P->pair ? 2 * TC_TILE_M : TC_TILE_M;
    P->choice.assign(P->count, BatchChoice{});
    for (int i = 0; i < P->count; i++) {
        const int64_t m = P->m[i], k = P->k[i], n = P->n[i];
        BatchChoice& c = P->choice[i];
        // CUDA cores: 128 x 128 tiles, k in 256-bit stages
        const int64_t pc_st = ceil_div(k, 256);
        const double pc_cost = (double)(ceil_div(m, POPC_TILE) * ceil_div(n, POPC_TILE)) *
                               (pc_st * M.pc_stage + M.pc_tile) / std::max(1, M.pc_units);
        double tc_cost = INFINITY;
        int64_t nks = 0;
        int n128 = 0;
        if (tc) {
            const int64_t kpad = ((k / 64 + 1) / 2 * 2) * 64;  // even word pitch
            nks = ceil_div(kpad, kst);
            const int64_t tn = ceil_div(n, TC_TILE_N);
            const int64_t tail = n - (tn - 1) * TC_TILE_N;
            n128 = (tail <= TC_TILE_N / 2 && M.tc_stage128 < M.tc_stage) ? 1 : 0;
            const double full = nks * M.tc_stage + M.tc_tile;
            const double half = nks * M.tc_stage128 + M.tc_tile;
            tc_cost = (double)ceil_div(m, tile_m) * ((tn - n128) * full + n128 * half) /
                      std::max(1, M.tc_units);
        }
        const int want = req ? req[i] : BMM_PATH_AUTO;
        // Strassen depth per shape (Sec. 3.8): the single-product planner's
        // choice (its rule: recurse while every leaf side stays >= 8192 bits,
        // or a tuned record for the shape); a binary product it gives depth
        // > 0 runs as its own Strassen product after the persistent launches.
        // AUTO entries of a plan on the device's automatic tensor path leave
        // the path to that planner too (a tuned record applies); otherwise
        // the entry's path, or the plan's tensor path, is fixed.
        if (P->op[i] == OP_GF2) {
            bmm_opts o;
            bmm_opts_default(&o);
            if (want != BMM_PATH_AUTO)
                o.path = want;
            else if (P->tc_path != auto_path())
                o.path = P->tc_path;
            Plan sp;
            if (make_plan(OP_GF2, m, k, n, &o, &sp) == BMM_OK && sp.depth > 0) {
                c.strassen = true;
                c.sp = sp;
                c.path = sp.path;
                continue;
            }
        }
        const bool use_tc = tc && (want == P->tc_path || (want == BMM_PATH_AUTO && tc_cost <= pc_cost));
        if (use_tc) {
            c.path = P->tc_path;
            c.n128 = n128;
            c.nks = nks;
            c.cost_ns = tc_cost * std::max(1, M.tc_units);
        } else {
            c.path = BMM_PATH_POPC;
            c.nks = pc_st;
            c.cost_ns = pc_cost * std::max(1, M.pc_units);
        }
    }
}

bmm_status plan_build(bmm_batched_plan_s* P) {
    const int count = P->count;
    const Model& M = P->model;
    const int tile_m = P->pair ? 2 * TC_TILE_M : TC_TILE_M;
    const int64_t kst = P->tc_path != BMM_PATH_POPC ? op_stage_bits(P->tc_path) : 256;
    // sizes of every device array
    std::vector<uint64_t> bt_off(count), ap_off(count, 0);
    P->kp.resize(count);
    uint64_t ws = 0;
    int pads = 0;
    P->tc_problems = P->pc_problems = 0;
    P->macs_needed = P->macs_issued = 0.0;
    uint64_t strassen_ws = 0;
    P->strassen_problems = 0;
    for (int i = 0; i < count; i++) {
        const int64_t kw = P->k[i] / 64;
        const bool tc = P->choice[i].path != BMM_PATH_POPC;
        P->kp[i] = (kw + 1) / 2 * 2;
        if (P->choice[i].strassen) {
            // its own plan's passes (transpose, XOR passes, leaves) in a
            // scratch shared with the other Strassen problems (they run one
            // after another)
            const Plan& sp = P->choice[i].sp;
            strassen_ws = std::max<uint64_t>(strassen_ws, sp.workspace_bytes);
            P->strassen_problems++;
            P->macs_needed += (double)P->m[i] * (double)P->k[i] * (double)P->n[i];
            double leaves = 1.0;
            for (int l = 0; l < sp.depth; l++) leaves *= 7.0;
            P->macs_issued += leaves * (double)(sp.m >> sp.depth) * (double)(sp.kp >> sp.depth) *
                              (double)(sp.n >> sp.depth);
            P->tc_problems += is_tc_path(sp.path) ? 1 : 0;
            P->pc_problems += is_tc_path(sp.path) ? 0 : 1;
            bt_off[i] = 0;
            continue;
        }
        bt_off[i] = ws;
        ws += round256((uint64_t)P->n[i] * P->kp[i] * 8);
        if (tc && (kw & 1)) {
            ap_off[i] = ws;
            ws += round256((uint64_t)P->m[i] * P->kp[i] * 8);
            pads++;
        }
        P->macs_needed += (double)P->m[i] * (double)P->k[i] * (double)P->n[i];
        if (tc) P->tc_problems++; else P->pc_problems++;
    }
    // tensor tiles and their LPT assignment (model cost of each tile)
    std::vector<TcWorkItem> items;
    std::vector<double> tile_cost;
    std::vector<PopcTile> ptiles;
    std::vector<double> ptile_cost;
    P->tc_tiles = P->tc_tiles128 = 0;
    for (int i = 0; i < count; i++) {
        const BatchChoice& c = P->choice[i];
        if (c.strassen) continue;
        if (c.path == BMM_PATH_POPC) {
            const int tm_n = (int)ceil_div(P->m[i], POPC_TILE), tn_n = (int)ceil_div(P->n[i], POPC_TILE);
            const double cost = c.nks * M.pc_stage + M.pc_tile;
            for (int a = 0; a < tm_n; a++)
                for (int b = 0; b < tn_n; b++) {
                    ptiles.push_back({i, a, b, 0});
                    ptile_cost.push_back(cost);
                }
            P->macs_issued += (double)tm_n * tn_n * POPC_TILE * POPC_TILE * (double)c.nks * 256.0;
            continue;
        }
        const int tm_n = (int)ceil_div(P->m[i], tile_m);
        const int tn_n = (int)ceil_div(P->n[i], TC_TILE_N);
        for (int a = 0; a < tm_n; a++)
            for (int b = 0; b < tn_n; b++) {
                TcWorkItem w;
                std::memset(&w, 0, sizeof(w));
                w.prob = i;
                w.tm = a;
                w.tn = b;
                w.nks = (int32_t)c.nks;
                w.n128 = (c.n128 && b == tn_n - 1) ? 1 : 0;
                w.op = P->op[i];
                w.m = (int32_t)P->m[i];
                w.n = (int32_t)P->n[i];
                w.C = P->C[i];
                w.ldc = P->n[i] / 64;
                items.push_back(w);
                tile_cost.push_back(c.nks * (w.n128 ? M.tc_stage128 : M.tc_stage) + M.tc_tile);
                P->tc_tiles++;
                P->tc_tiles128 += w.n128;
                P->macs_issued +=
                    (double)tile_m * (w.n128 ? TC_TILE_N / 2 : TC_TILE_N) * (double)c.nks * kst;
            }
    }
    const int slots = P->tc_path == BMM_PATH_POPC ? 0 : M.tc_units;
    const int grid = items.empty() ? 0 : (int)std::min<int64_t>((int64_t)items.size(), slots);
    std::vector<size_t> order(items.size());
    for (size_t t = 0; t < order.size(); t++) order[t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return tile_cost[x] > tile_cost[y]; });
    std::vector<std::vector<TcWorkItem>> per(grid);
    double makespan = 0.0;
    if (grid > 0) {
        using Load = std::pair<double, int>;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int c = 0; c < grid; c++) heap.push({0.0, c});
        for (size_t t : order) {
            Load l = heap.top();
            heap.pop();
            per[l.second].push_back(items[t]);
            l.first += tile_cost[t];
            heap.push(l);
        }
        while (!heap.empty()) {
            makespan = std::max(makespan, heap.top().first);
            heap.pop();
        }
    }
    // item offsets per unit, then each unit's packed stages (the kernel's
    // roles size their loops by it without walking the list)
    std::vector<int32_t> cta_ptr(2 * (grid + 1), 0);
    std::vector<TcWorkItem> flat;
    flat.reserve(items.size());
    for (int c = 0; c < grid; c++) {
        cta_ptr[c] = (int32_t)flat.size();
        int64_t pits = 0;
        for (const TcWorkItem& w : per[c]) {
            flat.push_back(w);
            pits += (w.nks + 1) / 2;
        }
        cta_ptr[grid + 1 + c] = (int32_t)pits;
    }
    cta_ptr[grid] = (int32_t)flat.size();
    P->grid = grid;
    // CUDA-core tiles longest first; the launch deals them out round robin
    std::vector<size_t> porder(ptiles.size());
    for (size_t t = 0; t < porder.size(); t++) porder[t] = t;
    std::stable_sort(porder.begin(), porder.end(),
                     [&](size_t x, size_t y) { return ptile_cost[x] > ptile_cost[y]; });
    std::vector<PopcTile> pflat;
    pflat.reserve(ptiles.size());
    double pc_makespan = 0.0;
    {
        const int units = std::max(1, M.pc_units);
        std::vector<double> load(units, 0.0);
        for (size_t j = 0; j < porder.size(); j++) {
            pflat.push_back(ptiles[porder[j]]);
            load[j % units] += ptile_cost[porder[j]];
        }
        for (double l : load) pc_makespan = std::max(pc_makespan, l);
    }
    P->pc_tiles = (int64_t)pflat.size();
    P->est_ms = (makespan + pc_makespan) * 1e-6;

    // one device allocation: workspace, then the tables
    const uint64_t off_sws = round256(ws);
    ws = off_sws + round256(strassen_ws);
    const uint64_t off_probs = round256(ws);
    const uint64_t off_items = round256(off_probs + sizeof(TcProblem) * (uint64_t)count);
    const uint64_t off_ptr = round256(off_items + sizeof(TcWorkItem) * flat.size());
    const uint64_t off_tjobs = round256(off_ptr + sizeof(int32_t) * 2 * (grid + 1));
    const uint64_t off_tfirst = round256(off_tjobs + sizeof(TransposeJob) * (uint64_t)count);
    const uint64_t off_pjobs = round256(off_tfirst + sizeof(int64_t) * (uint64_t)(count + 1));
    const uint64_t off_pfirst = round256(off_pjobs + sizeof(PadJob) * (uint64_t)std::max(pads, 1));
    const uint64_t off_pcjobs = round256(off_pfirst + sizeof(int64_t) * (uint64_t)(pads + 1));
    const uint64_t off_pctiles = round256(off_pcjobs + sizeof(PopcJob) * (uint64_t)count);
    const uint64_t off_ttjobs = round256(off_pctiles + sizeof(PopcTile) * (pflat.size() + 1));
    const uint64_t off_ttfirst = round256(off_ttjobs + sizeof(TmaTransposeJob) * (uint64_t)count);
    const uint64_t total = round256(off_ttfirst + sizeof(int64_t) * (uint64_t)(count + 1));
    BMM_CUDA_TRY(cudaMalloc(&P->dmem, total));
    char* base = (char*)P->dmem;
    P->d_probs = (TcProblem*)(base + off_probs);
    P->d_items = (TcWorkItem*)(base + off_items);
    P->d_cta_ptr = (int32_t*)(base + off_ptr);
    P->d_tjobs = (TransposeJob*)(base + off_tjobs);
    P->d_tfirst = (int64_t*)(base + off_tfirst);
    P->d_pjobs = (PadJob*)(base + off_pjobs);
    P->d_pfirst = (int64_t*)(base + off_pfirst);
    P->d_pcjobs = (PopcJob*)(base + off_pcjobs);
    P->d_pctiles = (PopcTile*)(base + off_pctiles);
    P->strassen_ws = strassen_ws ? (void*)(base + off_sws) : nullptr;
    P->d_ttjobs = (TmaTransposeJob*)(base + off_ttjobs);
    P->d_ttfirst = (int64_t*)(base + off_ttfirst);

    std::vector<TcProblem> probs(count);
    std::vector<TransposeJob> tjobs;
    std::vector<int64_t> tfirst(1, 0);
    std::vector<TmaTransposeJob> ttjobs;
    std::vector<int64_t> ttfirst(1, 0);
    std::vector<PadJob> pjobs;
    std::vector<int64_t> pfirst(1, 0);
    std::vector<PopcJob> pcjobs(count);
    P->Bt.resize(count);
    for (int i = 0; i < count; i++) {
        const int64_t kw = P->k[i] / 64;
        const bool tc = P->choice[i].path != BMM_PATH_POPC;
        std::memset(&probs[i], 0, sizeof(TcProblem));
        std::memset(&pcjobs[i], 0, sizeof(PopcJob));
        if (P->choice[i].strassen) {
            P->Bt[i] = nullptr;
            continue;
        }
        uint64_t* Bt = (uint64_t*)(base + bt_off[i]);
        P->Bt[i] = Bt;
        const uint64_t* Aop = P->A[i];
        int64_t lda = kw;
        if (tc && (kw & 1)) {
            uint64_t* Apad = (uint64_t*)(base + ap_off[i]);
            const int64_t ga = P->kp[i] <= 16 ? 32 / P->kp[i] : 1;
            const int64_t a_items = (P->m[i] + ga - 1) / ga;
            pjobs.push_back({P->A[i], Apad, Bt, P->m[i], P->n[i], kw, P->kp[i], ga, a_items});
            pfirst.push_back(pfirst.back() + a_items + (P->n[i] + 31) / 32);
            Aop = Apad;
            lda = P->kp[i];
        }
        if (tc) {
            const int64_t kpad = P->kp[i] * 64;
            if (!tc_make_problem(&probs[i], Aop, lda, Bt, P->kp[i], P->C[i], P->n[i] / 64, P->m[i],
                                 kpad, P->n[i], P->op[i], P->pair, P->fp4))
                return BMM_ERR_CUDA;
            probs[i].nks = (int32_t)P->choice[i].nks;
        }
        pcjobs[i] = {P->A[i], Bt, P->C[i], kw, P->kp[i], P->n[i] / 64,
                     P->m[i], P->k[i], P->n[i], P->op[i], 0};
        // B^T through the TMA form where its pitches allow, else load/store
        const TransposeJob tj = {P->B[i], Bt, P->n[i] / 64, P->kp[i], P->k[i], P->n[i]};
        TmaTransposeJob tt;
        std::memset(&tt, 0, sizeof(tt));
        if (make_transpose_tma_job(&tt, tj)) {
            ttjobs.push_back(tt);
            ttfirst.push_back(ttfirst.back() + transpose_tiles(P->k[i], P->n[i]));
        } else {
            tjobs.push_back(tj);
            tfirst.push_back(tfirst.back() + transpose_tiles(P->k[i], P->n[i]));
        }
    }
    P->transpose_count = (int)tjobs.size();
    P->transpose_total = tfirst.back();
    P->tma_count = (int)ttjobs.size();
    P->tma_total = ttfirst.back();
    P->pad_count = pads;
    P->pad_total = pfirst.back();
    if (count > 0)
        BMM_CUDA_TRY(cudaMemcpy(P->d_probs, probs.data(), sizeof(TcProblem) * count,
                                cudaMemcpyHostToDevice));
    if (!flat.empty())
        BMM_CUDA_TRY(cudaMemcpy(P->d_items, flat.data(), sizeof(TcWorkItem) * flat.size(),
                                cudaMemcpyHostToDevice));
    BMM_CUDA_TRY(cudaMemcpy(P->d_cta_ptr, cta_ptr.data(), sizeof(int32_t) * 2 * (grid + 1),
                            cudaMemcpyHostToDevice));
    if (!tjobs.empty()) {
        BMM_CUDA_TRY(cudaMemcpy(P->d_tjobs, tjobs.data(), sizeof(TransposeJob) * tjobs.size(),
                                cudaMemcpyHostToDevice));
        BMM_CUDA_TRY(cudaMemcpy(P->d_tfirst, tfirst.data(), sizeof(int64_t) * tjobs.size(),
                                cudaMemcpyHostToDevice));
    }
    if (!ttjobs.empty()) {
        BMM_CUDA_TRY(cudaMemcpy(P->d_ttjobs, ttjobs.data(), sizeof(TmaTransposeJob) * ttjobs.size(),
                                cudaMemcpyHostToDevice));
        BMM_CUDA_TRY(cudaMemcpy(P->d_ttfirst, ttfirst.data(), sizeof(int64_t) * ttjobs.size(),
                                cudaMemcpyHostToDevice));
    }
    if (pads) {
        BMM_CUDA_TRY(cudaMemcpy(P->d_pjobs, pjobs.data(), sizeof(PadJob) * pads,
                                cudaMemcpyHostToDevice));
        BMM_CUDA_TRY(cudaMemcpy(P->d_pfirst, pfirst.data(), sizeof(int64_t) * pads,
                                cudaMemcpyHostToDevice));
    }
    if (count > 0)
        BMM_CUDA_TRY(cudaMemcpy(P->d_pcjobs, pcjobs.data(), sizeof(PopcJob) * count,
                                cudaMemcpyHostToDevice));
    if (!pflat.empty())
        BMM_CUDA_TRY(cudaMemcpy(P->d_pctiles, pflat.data(), sizeof(PopcTile) * pflat.size(),
                                cudaMemcpyHostToDevice));
    return BMM_OK;
}

// The base-case launches of a plan (the tensor tiles, then the CUDA-core ones).
bmm_status plan_run_base(bmm_batched_plan_s* P, cudaStream_t s) {
    if (P->grid > 0)
        BMM_CUDA_TRY(tc_launch_batched(P->d_probs, P->d_items, P->d_cta_ptr, P->grid, P->pair,
                                       P->fp4, s));
    if (P->pc_tiles > 0) BMM_CUDA_TRY(launch_popc_batched(P->d_pcjobs, P->d_pctiles, P->pc_tiles, s));
    return BMM_OK;
}

bmm_status plan_run(bmm_batched_plan_s* P, cudaStream_t s) {
    if (P->count == 0) return BMM_OK;
    BMM_CUDA_TRY(launch_transpose_tma_batched(P->d_ttjobs, P->d_ttfirst, P->tma_count,
                                              P->tma_total, s));
    BMM_CUDA_TRY(launch_transpose_batched(P->d_tjobs, P->d_tfirst, P->transpose_count,
                                          P->transpose_total, s));
    if (P->pad_count) {
        const int64_t warps = P->pad_total;
        int64_t blocks = (warps * 32 + 255) / 256;
        const int64_t cap = (int64_t)sm_count() * 16;
        if (blocks > cap) blocks = cap;
        TraceScope ts(BMM_PHASE_TRANSPOSE, s);
        pad_kernel<<<(unsigned)blocks, 256, 0, s>>>(P->d_pjobs, P->d_pfirst, P->pad_count,
                                                    P->pad_total);
        BMM_CUDA_TRY(cudaGetLastError());
    }
    bmm_status st = plan_run_base(P, s);
    if (st != BMM_OK) return st;
    for (int i = 0; i < P->count; i++)
        if (P->choice[i].strassen) {
            st = execute_plan(P->choice[i].sp, P->A[i], P->B[i], P->C[i], P->strassen_ws, s);
            if (st != BMM_OK) return st;
        }
    return BMM_OK;
}

void plan_free(bmm_batched_plan_s* P) {
    if (P->dmem) cudaFree(P->dmem);
    delete P;
}

// A plan over the given problems with every choice fixed by `req` (no model
// measurement): the building block of the measurement itself.
bmm_status plan_fixed(int tc_path, const Model& M, std::vector<int64_t> ms, std::vector<int64_t> ks,
                      std::vector<int64_t> ns, const uint64_t* A, const uint64_t* B, uint64_t* C,
                      uint64_t c_stride_words, const std::vector<int32_t>& req,
                      bmm_batched_plan_s** out) {
    bmm_batched_plan_s* P = new bmm_batched_plan_s();
    cudaGetDevice(&P->device);
    P->count = (int)ms.size();
    P->tc_path = tc_path;
    P->fp4 = tc_path == BMM_PATH_TC_FP4_PAIR;
    P->pair = tc_path == BMM_PATH_TC_FP4_PAIR || tc_path == BMM_PATH_TC_FP8_PAIR;
    P->model = M;
    P->op.assign(P->count, OP_GF2);
    P->A.assign(P->count, A);
    P->B.assign(P->count, B);
    for (int i = 0; i < P->count; i++) P->C.push_back(C + (uint64_t)i * c_stride_words);
    P->m = std::move(ms);
    P->k = std::move(ks);
    P->n = std::move(ns);
    decide(P, req.data());
    const bmm_status st = plan_build(P);
    if (st != BMM_OK) {
        plan_free(P);
        return st;
    }
    *out = P;
    return BMM_OK;
}

// Best of three base-case runs (after one whole run), milliseconds.
bmm_status time_base(bmm_batched_plan_s* P, cudaStream_t s, double* ms) {
    cudaEvent_t a, b;
    BMM_CUDA_TRY(cudaEventCreate(&a));
    BMM_CUDA_TRY(cudaEventCreate(&b));
    bmm_status st = plan_run(P, s);
    double best = INFINITY;
    for (int r = 0; st == BMM_OK && r < 3; r++) {
        cudaEventRecord(a, s);
        st = plan_run_base(P, s);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) st = BMM_ERR_CUDA;
        float t = 0.f;
        if (st == BMM_OK && cudaEventElapsedTime(&t, a, b) == cudaSuccess) best = std::min(best, (double)t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return st;
}

// Largest number of tiles one unit of the plan runs (tensor or CUDA-core).
double busiest_tc(const bmm_batched_plan_s* P) {
    const int64_t tiles = P->tc_tiles;
    return (double)ceil_div(tiles, std::max(1, P->grid));
}
double busiest_pc(const bmm_batched_plan_s* P, int units) {
    return (double)ceil_div(P->pc_tiles, std::max(1, units));
}

// Measures the model on the current device (synthetic batches of equal
// problems, operands of arbitrary content: the time does not depend on it).
bmm_status measure_model(int tc_path, Model* out) {
    Model M = default_model(tc_path);
    const bool tc = tc_path != BMM_PATH_POPC;
    if (tc) M.tc_units = tc_path == BMM_PATH_TC_FP8 ? sm_count() : tc_pair_slots(tc_path == BMM_PATH_TC_FP4_PAIR);
    M.pc_units = popc_batched_grid();
    // problems of 2048 x k x 2048 (k = 4096 and 256): 64 tensor tiles each on
    // SM pairs (128 on single SMs), 256 CUDA-core tiles; about 32 tensor
    // tiles per unit. The N = 128 batch has n = 128 and 8 times as many.
    const int64_t S = 2048, K = 4096, Kshort = 256;
    const int64_t tiles_per = (S / (tc && tc_path == BMM_PATH_TC_FP8 ? TC_TILE_M : 2 * TC_TILE_M)) *
                              (S / TC_TILE_N);
    const int nprob = (int)std::max<int64_t>(8, ceil_div(32 * (int64_t)std::max(1, M.tc_units), tiles_per));
    const int nnarrow = 8 * nprob;
    void* mem = nullptr;
    const uint64_t a_words = (uint64_t)S * K / 64, b_words = (uint64_t)K * S / 64;
    const uint64_t c_words = (uint64_t)S * S / 64;
    const uint64_t c128_words = (uint64_t)S * 128 / 64;
    const uint64_t total_words = a_words + b_words + std::max<uint64_t>(c_words * nprob, c128_words * nnarrow);
    BMM_CUDA_TRY(cudaMalloc(&mem, total_words * 8));
    uint64_t* A = (uint64_t*)mem;
    uint64_t* B = A + a_words;
    uint64_t* C = B + b_words;
    cudaStream_t s = nullptr;
    bmm_status st = BMM_OK;
    if (cudaMemset(mem, 0x5A, (a_words + b_words) * 8) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        st = BMM_ERR_CUDA;
    auto run = [&](int path, int64_t m, int64_t k, int64_t n, int cnt, uint64_t cstride, double* ms,
                   double* busiest) -> bmm_status {
        bmm_batched_plan_s* P = nullptr;
        bmm_status r = plan_fixed(tc ? tc_path : BMM_PATH_POPC, M, std::vector<int64_t>(cnt, m),
                                  std::vector<int64_t>(cnt, k), std::vector<int64_t>(cnt, n), A, B,
                                  C, cstride, std::vector<int32_t>(cnt, path), &P);
        if (r != BMM_OK) return r;
        r = time_base(P, s, ms);
        *busiest = path == BMM_PATH_POPC ? busiest_pc(P, M.pc_units) : busiest_tc(P);
        plan_free(P);
        return r;
    };
    if (st == BMM_OK && tc) {
        // long and short k (operand stages o1 > o2), then N = 128 at long k
        const int64_t kst = op_stage_bits(tc_path);
        const double o1 = (double)ceil_div(K, kst), o2 = (double)ceil_div(Kshort, kst);
        double t1 = 0, t2 = 0, t3 = 0, b1 = 1, b2 = 1, b3 = 1;
        // (the default model's N = 128 stage is the cheaper one, so every
        // tile of the n = 128 batch runs N = 128)
        st = run(tc_path, S, K, S, nprob, c_words, &t1, &b1);
        if (st == BMM_OK) st = run(tc_path, S, Kshort, S, nprob, c_words, &t2, &b2);
        if (st == BMM_OK) st = run(tc_path, S, K, 128, nnarrow, c128_words, &t3, &b3);
        if (st == BMM_OK) {
            const double per1 = t1 * 1e6 / b1, per2 = t2 * 1e6 / b2, per3 = t3 * 1e6 / b3;
            const double stage = (per1 - per2) / (o1 - o2);
            if (stage > 0 && std::isfinite(stage)) {
                M.tc_stage = stage;
                M.tc_tile = std::max(0.0, per2 - o2 * stage);
                M.tc_stage128 = std::max(0.0, (per3 - M.tc_tile) / o1);
            }
        }
    }
    if (st == BMM_OK) {
        const double o1 = (double)ceil_div(K, 256), o2 = (double)ceil_div(Kshort, 256);
        double t1 = 0, t2 = 0, b1 = 1, b2 = 1;
        st = run(BMM_PATH_POPC, S, K, S, nprob, c_words, &t1, &b1);
        if (st == BMM_OK) st = run(BMM_PATH_POPC, S, Kshort, S, nprob, c_words, &t2, &b2);
        if (st == BMM_OK) {
            const double per1 = t1 * 1e6 / b1, per2 = t2 * 1e6 / b2;
            const double stage = (per1 - per2) / (o1 - o2);
            if (stage > 0 && std::isfinite(stage)) {
                M.pc_stage = stage;
                M.pc_tile = std::max(0.0, per2 - o2 * stage);
            }
        }
    }
    if (s) cudaStreamDestroy(s);
    cudaFree(mem);
    if (st != BMM_OK) return st;
    // A measurement disturbed from outside (another process on the GPU, a
    // profiler serialising launches) gives figures far from any this kernel
    // has: keep the built-in ones then, and measure again on a later plan.
    const Model D = default_model(tc_path);
    auto plausible = [](double v, double ref) { return v >= ref / 8.0 && v <= ref * 8.0; };
    if ((tc && !(plausible(M.tc_stage, D.tc_stage) && plausible(M.tc_stage128, D.tc_stage128) &&
                 plausible(M.tc_tile + D.tc_stage, D.tc_tile + D.tc_stage))) ||
        !(plausible(M.pc_stage, D.pc_stage) && plausible(M.pc_tile + D.pc_stage, D.pc_tile + D.pc_stage)))
        return BMM_ERR_CUDA;
    M.measured = true;
    *out = M;
    return BMM_OK;
}

// The measured model for (device, tensor path), measured on first use.
std::mutex g_model_mu;
bmm_status model_for(int tc_path, Model* out) {
    static Model cache[64][6];
    static bool have[64][6] = {{false}};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64 || tc_path < 0 || tc_path > 5) {
        *out = default_model(tc_path);
        return BMM_OK;
    }
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!have[d][tc_path]) {
        Model M;
        if (measure_model(tc_path, &M) != BMM_OK) {
            // no room or no time to measure now: decide with the built-in
            // figures (reported as not measured) and measure on a later plan
            (void)cudaGetLastError();
            *out = default_model(tc_path);
            return BMM_OK;
        }
        cache[d][tc_path] = M;
        have[d][tc_path] = true;
    }
    *out = cache[d][tc_path];
    return BMM_OK;
}

bmm_status check_batch(int32_t count, const int32_t* ops, const uint64_t* const* A,
                       const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                       const int64_t* k, const int64_t* n) {
    if (count < 0 || (count > 0 && (!ops || !A || !B || !C || !m || !k || !n)))
        return BMM_ERR_INVALID;
    for (int i = 0; i < count; i++) {
        if (ops[i] != OP_GF2 && ops[i] != OP_BOOL) return BMM_ERR_INVALID;
        if (!A[i] || !B[i] || !C[i]) return BMM_ERR_INVALID;
        if (m[i] <= 0 || k[i] <= 0 || n[i] <= 0 || m[i] % 64 || k[i] % 64 || n[i] % 64)
            return BMM_ERR_INVALID;
        if (((uintptr_t)A[i] | (uintptr_t)B[i] | (uintptr_t)C[i]) & 15u) return BMM_ERR_ALIGN;
        if (m[i] > 0x7fffffff || n[i] > 0x7fffffff) return BMM_ERR_UNSUPPORTED;
    }
    return BMM_OK;
}

// paths: per problem AUTO, BMM_PATH_POPC or one tensor path (the same for
// every tensor entry), or nullptr with `path` for all of them.
bmm_status plan_create(int32_t count, const int32_t* ops, const uint64_t* const* A,
                       const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                       const int64_t* k, const int64_t* n, int32_t path, const int32_t* paths,
                       bmm_batched_plan* plan) {
    if (!plan) return BMM_ERR_INVALID;
    *plan = nullptr;
    bmm_status st = check_batch(count, ops, A, B, C, m, k, n);
    if (st != BMM_OK) return st;
    // the plan's tensor path: the one named, else the device's automatic one
    int tcp = BMM_PATH_AUTO;
    std::vector<int32_t> req(count > 0 ? count : 0, path);
    if (paths) {
        for (int i = 0; i < count; i++) {
            const int p = paths[i];
            if (p == BMM_PATH_TC_I8) return BMM_ERR_UNSUPPORTED;
            if (p != BMM_PATH_AUTO && p != BMM_PATH_POPC && !is_tc_path(p)) return BMM_ERR_INVALID;
            if (is_tc_path(p)) {
                if (tcp != BMM_PATH_AUTO && tcp != p) return BMM_ERR_INVALID;
                tcp = p;
            }
            req[i] = p;
        }
    } else {
        if (path == BMM_PATH_TC_I8) return BMM_ERR_UNSUPPORTED;
        if (path != BMM_PATH_AUTO && path != BMM_PATH_POPC && !is_tc_path(path))
            return BMM_ERR_INVALID;
        if (is_tc_path(path)) tcp = path;
    }
    bool all_popc = !paths && path == BMM_PATH_POPC;
    if (paths) {
        all_popc = true;
        for (int i = 0; i < count; i++) all_popc = all_popc && paths[i] == BMM_PATH_POPC;
    }
    if (tcp == BMM_PATH_AUTO) tcp = all_popc ? BMM_PATH_POPC : auto_path();
    if (is_tc_path(tcp)) {
        if (!tc_path_available()) return BMM_ERR_UNSUPPORTED;
        if (tcp != BMM_PATH_TC_FP8 && tc_pair_slots(tcp == BMM_PATH_TC_FP4_PAIR) <= 0)
            return BMM_ERR_UNSUPPORTED;
    }
    bmm_batched_plan_s* P = new bmm_batched_plan_s();
    cudaGetDevice(&P->device);
    P->count = count;
    P->tc_path = tcp;
    P->fp4 = tcp == BMM_PATH_TC_FP4_PAIR;
    P->pair = tcp == BMM_PATH_TC_FP4_PAIR || tcp == BMM_PATH_TC_FP8_PAIR;
    P->op.assign(ops, ops + count);
    P->A.assign(A, A + count);
    P->B.assign(B, B + count);
    P->C.assign(C, C + count);
    P->m.assign(m, m + count);
    P->k.assign(k, k + count);
    P->n.assign(n, n + count);
    // the measured model decides whatever is left open (paths, tail tiles)
    st = count > 0 ? model_for(tcp, &P->model) : BMM_OK;
    if (st == BMM_OK) {
        decide(P, req.data());
        st = plan_build(P);
    }
    // what the first run would otherwise set up (the device error word, the
    // kernel attributes), so that even a plan's first run can be captured
    if (st == BMM_OK && count > 0 && !device_error_word()) st = BMM_ERR_NOMEM;
    if (st == BMM_OK && P->grid > 0) {
        const cudaError_t e = tc_prepare_batched(P->pair, P->fp4);
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (st != BMM_OK) {
        plan_free(P);
        return st;
    }
    *plan = P;
    return BMM_OK;
}

}  // namespace

extern "C" {

bmm_status bmm_batched_plan_create(int32_t count, const int32_t* ops, const uint64_t* const* A,
                                   const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                                   const int64_t* k, const int64_t* n, bmm_batched_plan* plan) {
    return plan_create(count, ops, A, B, C, m, k, n, BMM_PATH_AUTO, nullptr, plan);
}

bmm_status bmm_batched_plan_create_ex(int32_t count, const int32_t* ops,
                                      const uint64_t* const* A, const uint64_t* const* B,
                                      uint64_t* const* C, const int64_t* m, const int64_t* k,
                                      const int64_t* n, int32_t path, bmm_batched_plan* plan) {
    return plan_create(count, ops, A, B, C, m, k, n, path, nullptr, plan);
}

bmm_status bmm_batched_plan_create_paths(int32_t count, const int32_t* ops,
                                         const uint64_t* const* A, const uint64_t* const* B,
                                         uint64_t* const* C, const int64_t* m, const int64_t* k,
                                         const int64_t* n, const int32_t* paths,
                                         bmm_batched_plan* plan) {
    if (count > 0 && !paths) return BMM_ERR_INVALID;
    return plan_create(count, ops, A, B, C, m, k, n, BMM_PATH_AUTO, paths, plan);
}

bmm_status bmm_batched_plan_run(bmm_batched_plan plan, bmm_stream_t stream) {
    if (!plan) return BMM_ERR_INVALID;
    return plan_run(plan, (cudaStream_t)stream);
}

bmm_status bmm_batched_plan_path(bmm_batched_plan plan, int32_t* path) {
    if (!plan || !path) return BMM_ERR_INVALID;
    *path = plan->tc_problems > 0 ? plan->tc_path : BMM_PATH_POPC;
    return BMM_OK;
}

bmm_status bmm_batched_plan_choice(bmm_batched_plan plan, int32_t i, bmm_batched_choice* out) {
    if (!plan || !out || i < 0 || i >= plan->count) return BMM_ERR_INVALID;
    const BatchChoice& c = plan->choice[i];
    std::memset(out, 0, sizeof(*out));
    out->path = c.path;
    out->strassen_depth = c.strassen ? c.sp.depth : 0;
    if (c.strassen) {
        // its own product: the base case's tile over the leaves
        const bool pair = c.path == BMM_PATH_TC_FP4_PAIR || c.path == BMM_PATH_TC_FP8_PAIR;
        out->tile_m = c.path == BMM_PATH_POPC ? POPC_TILE : pair ? 2 * TC_TILE_M : TC_TILE_M;
        out->tile_n = out->tail_n = c.path == BMM_PATH_POPC ? POPC_TILE : TC_TILE_N;
        out->k_step = c.path == BMM_PATH_POPC ? 256 : (int32_t)op_stage_bits(c.path);
        out->k_steps = ceil_div(c.sp.kp >> c.sp.depth, out->k_step);
        out->est_us = 0.0;
        return BMM_OK;
    }
    if (c.path == BMM_PATH_POPC) {
        out->tile_m = out->tile_n = out->tail_n = POPC_TILE;
        out->k_step = 256;
    } else {
        out->tile_m = plan->pair ? 2 * TC_TILE_M : TC_TILE_M;
        out->tile_n = TC_TILE_N;
        out->tail_n = c.n128 ? TC_TILE_N / 2 : TC_TILE_N;
        out->k_step = (int32_t)op_stage_bits(c.path);
    }
    out->k_steps = c.nks;
    out->est_us = c.cost_ns * 1e-3;
    return BMM_OK;
}

bmm_status bmm_batched_plan_stats(bmm_batched_plan plan, bmm_batched_stats* out) {
    if (!plan || !out) return BMM_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    out->problems = plan->count;
    out->tensor_problems = plan->tc_problems;
    out->popc_problems = plan->pc_problems;
    out->tensor_tiles = plan->tc_tiles;
    out->tensor_tiles_n128 = plan->tc_tiles128;
    out->popc_tiles = plan->pc_tiles;
    out->macs_needed = plan->macs_needed;
    out->macs_issued = plan->macs_issued;
    out->est_ms = plan->est_ms;
    out->model_measured = plan->model.measured ? 1 : 0;
    out->tensor_path = plan->tc_path;
    out->strassen_problems = plan->strassen_problems;
    return BMM_OK;
}

bmm_status bmm_batched_model(int32_t path, bmm_batched_model_info* out) {
    if (!out) return BMM_ERR_INVALID;
    if (path == BMM_PATH_AUTO) path = auto_path();
    if (path == BMM_PATH_TC_I8) return BMM_ERR_UNSUPPORTED;
    if (path != BMM_PATH_POPC && !is_tc_path(path)) return BMM_ERR_INVALID;
    if (is_tc_path(path) && !tc_path_available()) return BMM_ERR_UNSUPPORTED;
    Model M;
    const bmm_status st = model_for(path, &M);
    if (st != BMM_OK) return st;
    std::memset(out, 0, sizeof(*out));
    out->path = path;
    out->measured = M.measured ? 1 : 0;
    out->tensor_units = M.tc_units;
    out->tensor_stage_ns = M.tc_stage;
    out->tensor_stage_n128_ns = M.tc_stage128;
    out->tensor_tile_ns = M.tc_tile;
    out->popc_units = M.pc_units;
    out->popc_stage_ns = M.pc_stage;
    out->popc_tile_ns = M.pc_tile;
    return BMM_OK;
}

bmm_status bmm_batched_plan_destroy(bmm_batched_plan plan) {
    if (!plan) return BMM_OK;
    cudaError_t e = cudaSuccess;
    if (plan->dmem) e = cudaFree(plan->dmem);
    delete plan;
    return e == cudaSuccess ? BMM_OK : cuda_fail(e);
}

bmm_status bmm_batched(int32_t count, const int32_t* ops, const uint64_t* const* A,
                       const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                       const int64_t* k, const int64_t* n, bmm_stream_t stream) {
    bmm_batched_plan plan = nullptr;
    bmm_status st = bmm_batched_plan_create(count, ops, A, B, C, m, k, n, &plan);
    if (st != BMM_OK) return st;
    st = bmm_batched_plan_run(plan, stream);
    // the plan's memory must outlive the launched work: wait, then free
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    const bmm_status sd = bmm_batched_plan_destroy(plan);
    if (st != BMM_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e);
    return sd;
}

}  // extern "C"

namespace bmm {

bmm_status run_batched(int op, int32_t count, const uint64_t* const* A, const uint64_t* const* B,
                       uint64_t* const* C, const int64_t* m, const int64_t* k, const int64_t* n,
                       cudaStream_t s) {
    if (count < 0) return BMM_ERR_INVALID;
    std::vector<int32_t> ops((size_t)count, op);
    return bmm_batched(count, ops.data(), A, B, C, m, k, n, s);
}

}  // namespace bmm
