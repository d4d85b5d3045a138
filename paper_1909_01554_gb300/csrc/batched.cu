// Batched products of uneven sizes in one persistent launch.
//
// A plan is built once on the host: per-problem TMA maps over A (or a copy of
// A with an even row pitch) and over the transposed B, the work list of all
// 256 x 256 output tiles (128 x 256 where SM pairs are unavailable), and a
// longest-processing-time-first assignment of the tiles to the resident CTA
// pairs (or CTAs); each tile costs its k stages plus a fixed epilogue share. Running a plan only launches kernels: one batched bit
// transpose of every B, one pass that pads rows whose k/64 word count is odd,
// and one persistent launch of the tensor-core base case that walks each
// CTA's list. Nothing in a run allocates or synchronises, so a run can be
// captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include "plan.h"
#include "tc_batched.h"

namespace bmm {

namespace {

constexpr int EPI_COST = 4;  // epilogue of one tile, in 128-bit k stages

// Rows of odd-k problems: copy A rows into the even-pitch buffer (zeroing the
// pad word) and zero the pad word of every Bt row. One warp per row.
struct PadJob {
    const uint64_t* A;
    uint64_t* Apad;
    uint64_t* Bt;
    int64_t m, n, kw, kp;  // kw = k/64 (odd), kp = kw + 1
};

__global__ void __launch_bounds__(256) pad_kernel(const PadJob* __restrict__ jobs,
                                                  const int64_t* __restrict__ first, int count,
                                                  int64_t total_rows) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < total_rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const PadJob j = jobs[lo];
        const int64_t local = r - first[lo];
        if (local < j.m) {
            const uint64_t* src = j.A + local * j.kw;
            uint64_t* dst = j.Apad + local * j.kp;
            for (int64_t w = lane; w < j.kp; w += 32) dst[w] = w < j.kw ? src[w] : 0ull;
        } else if (lane == 0) {
            j.Bt[(local - j.m) * j.kp + j.kw] = 0ull;
        }
    }
}

uint64_t round256(uint64_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace bmm

using namespace bmm;

struct bmm_batched_plan_s {
    int device = 0;
    int count = 0;
    bool tc = false;
    bool pair = false;  // SM pairs: 256-row tiles, one work list per CTA pair
    bool fp4 = false;   // e2m1 operands (SM pairs only)
    // problem list (host)
    std::vector<int> op;
    std::vector<const uint64_t*> A, B;
    std::vector<uint64_t*> C;
    std::vector<int64_t> m, k, n;
    // device memory owned by the plan (one allocation)
    void* dmem = nullptr;
    TcProblem* d_probs = nullptr;
    TcWorkItem* d_items = nullptr;
    int32_t* d_cta_ptr = nullptr;
    TransposeJob* d_tjobs = nullptr;
    int64_t* d_tfirst = nullptr;
    PadJob* d_pjobs = nullptr;
    int64_t* d_pfirst = nullptr;
    int grid = 0;
    int64_t transpose_total = 0, pad_total = 0;
    int pad_count = 0;
    std::vector<uint64_t*> Bt;  // per problem, inside dmem
    std::vector<int64_t> kp;
};

namespace {

// path: the base case every problem runs on (resolved, never AUTO).
bmm_status plan_build(bmm_batched_plan_s* P, int path) {
    const int count = P->count;
    P->tc = is_tc_path(path);
    P->fp4 = path == BMM_PATH_TC_FP4_PAIR;
    const int pair_slots =
        path == BMM_PATH_TC_FP8 ? 0 : P->tc ? tc_pair_slots(P->fp4) : 0;
    if (path != BMM_PATH_TC_FP8 && P->tc && pair_slots <= 0) return BMM_ERR_UNSUPPORTED;
    P->pair = pair_slots > 0;
    const int tile_m = P->pair ? 2 * TC_TILE_M : TC_TILE_M;
    // sizes of every device array
    std::vector<uint64_t> bt_off(count), ap_off(count, 0);
    P->kp.resize(count);
    uint64_t ws = 0;
    int pads = 0;
    for (int i = 0; i < count; i++) {
        const int64_t kw = P->k[i] / 64;
        P->kp[i] = (kw + 1) / 2 * 2;
        bt_off[i] = ws;
        ws += round256((uint64_t)P->n[i] * P->kp[i] * 8);
        if (kw & 1) {
            ap_off[i] = ws;
            ws += round256((uint64_t)P->m[i] * P->kp[i] * 8);
            pads++;
        }
    }
    // tiles and their LPT assignment (cost: k stages plus an epilogue share)
    std::vector<TcWorkItem> items;
    std::vector<int32_t> cost_of(count);
    for (int i = 0; i < count; i++) {
        const int tm_n = (int)((P->m[i] + tile_m - 1) / tile_m);
        const int tn_n = (int)((P->n[i] + TC_TILE_N - 1) / TC_TILE_N);
        // cost: k in 128-bit units (the e2m1 form's stages carry twice the k
        // for about the same time, as far as the tensor rate allows)
        const int kstage = P->fp4 ? 512 : 256;
        // the padded k the problem's maps are built with (tc_make_problem)
        const int64_t kpad = P->kp[i] * 64;
        const int nks = (int)((kpad + kstage - 1) / kstage) * 2;
        for (int a = 0; a < tm_n; a++)
            for (int b = 0; b < tn_n; b++) items.push_back({i, a, b, nks});
        cost_of[i] = nks + EPI_COST;
    }
    const int slots = P->pair ? pair_slots : sm_count();
    const int grid = (int)std::min<int64_t>((int64_t)items.size(), slots);  // work units
    std::stable_sort(items.begin(), items.end(),
                     [&](const TcWorkItem& x, const TcWorkItem& y) {
                         return cost_of[x.prob] > cost_of[y.prob];
                     });
    std::vector<std::vector<TcWorkItem>> per(grid);
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < grid; c++) heap.push({0, c});
    for (const TcWorkItem& w : items) {
        Load l = heap.top();
        heap.pop();
        per[l.second].push_back(w);
        l.first += cost_of[w.prob];
        heap.push(l);
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

    // one device allocation: workspace, then the tables
    const uint64_t off_probs = round256(ws);
    const uint64_t off_items = round256(off_probs + sizeof(TcProblem) * (uint64_t)count);
    const uint64_t off_ptr = round256(off_items + sizeof(TcWorkItem) * flat.size());
    const uint64_t off_tjobs = round256(off_ptr + sizeof(int32_t) * 2 * (grid + 1));
    const uint64_t off_tfirst = round256(off_tjobs + sizeof(TransposeJob) * (uint64_t)count);
    const uint64_t off_pjobs = round256(off_tfirst + sizeof(int64_t) * (uint64_t)(count + 1));
    const uint64_t off_pfirst = round256(off_pjobs + sizeof(PadJob) * (uint64_t)std::max(pads, 1));
    const uint64_t total = round256(off_pfirst + sizeof(int64_t) * (uint64_t)(pads + 1));
    BMM_CUDA_TRY(cudaMalloc(&P->dmem, total));
    char* base = (char*)P->dmem;
    P->d_probs = (TcProblem*)(base + off_probs);
    P->d_items = (TcWorkItem*)(base + off_items);
    P->d_cta_ptr = (int32_t*)(base + off_ptr);
    P->d_tjobs = (TransposeJob*)(base + off_tjobs);
    P->d_tfirst = (int64_t*)(base + off_tfirst);
    P->d_pjobs = (PadJob*)(base + off_pjobs);
    P->d_pfirst = (int64_t*)(base + off_pfirst);

    std::vector<TcProblem> probs(count);
    std::vector<TransposeJob> tjobs(count);
    std::vector<int64_t> tfirst(count + 1, 0);
    std::vector<PadJob> pjobs;
    std::vector<int64_t> pfirst(1, 0);
    P->Bt.resize(count);
    for (int i = 0; i < count; i++) {
        const int64_t kw = P->k[i] / 64;
        uint64_t* Bt = (uint64_t*)(base + bt_off[i]);
        P->Bt[i] = Bt;
        const uint64_t* Aop = P->A[i];
        int64_t lda = kw;
        if (kw & 1) {
            uint64_t* Apad = (uint64_t*)(base + ap_off[i]);
            pjobs.push_back({P->A[i], Apad, Bt, P->m[i], P->n[i], kw, P->kp[i]});
            pfirst.push_back(pfirst.back() + P->m[i] + P->n[i]);
            Aop = Apad;
            lda = P->kp[i];
        }
        std::memset(&probs[i], 0, sizeof(TcProblem));
        if (P->tc) {
            const int64_t kpad = P->kp[i] * 64;
            if (!tc_make_problem(&probs[i], Aop, lda, Bt, P->kp[i], P->C[i], P->n[i] / 64, P->m[i],
                                 kpad, P->n[i], P->op[i], P->pair, P->fp4))
                return BMM_ERR_CUDA;
        }
        tjobs[i] = {P->B[i], Bt, P->n[i] / 64, P->kp[i], P->k[i], P->n[i]};
        tfirst[i + 1] = tfirst[i] + transpose_tiles(P->k[i], P->n[i]);
    }
    P->transpose_total = tfirst[count];
    P->pad_count = pads;
    P->pad_total = pfirst.back();
    BMM_CUDA_TRY(cudaMemcpy(P->d_probs, probs.data(), sizeof(TcProblem) * count,
                            cudaMemcpyHostToDevice));
    if (!flat.empty())
        BMM_CUDA_TRY(cudaMemcpy(P->d_items, flat.data(), sizeof(TcWorkItem) * flat.size(),
                                cudaMemcpyHostToDevice));
    BMM_CUDA_TRY(cudaMemcpy(P->d_cta_ptr, cta_ptr.data(), sizeof(int32_t) * 2 * (grid + 1),
                            cudaMemcpyHostToDevice));
    BMM_CUDA_TRY(cudaMemcpy(P->d_tjobs, tjobs.data(), sizeof(TransposeJob) * count,
                            cudaMemcpyHostToDevice));
    BMM_CUDA_TRY(cudaMemcpy(P->d_tfirst, tfirst.data(), sizeof(int64_t) * count,
                            cudaMemcpyHostToDevice));
    if (pads) {
        BMM_CUDA_TRY(cudaMemcpy(P->d_pjobs, pjobs.data(), sizeof(PadJob) * pads,
                                cudaMemcpyHostToDevice));
        BMM_CUDA_TRY(cudaMemcpy(P->d_pfirst, pfirst.data(), sizeof(int64_t) * pads,
                                cudaMemcpyHostToDevice));
    }
    return BMM_OK;
}

bmm_status plan_run(bmm_batched_plan_s* P, cudaStream_t s) {
    if (P->count == 0) return BMM_OK;
    BMM_CUDA_TRY(launch_transpose_batched(P->d_tjobs, P->d_tfirst, P->count, P->transpose_total, s));
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
    if (P->tc) {
        BMM_CUDA_TRY(tc_launch_batched(P->d_probs, P->d_items, P->d_cta_ptr, P->grid, P->pair, P->fp4, s));
        return BMM_OK;
    }
    // without tensor cores: the CUDA-core base case, one launch per problem
    for (int i = 0; i < P->count; i++) {
        bmm_status st = run_base_product(P->op[i], BMM_PATH_POPC, P->A[i], P->k[i] / 64, P->Bt[i],
                                         P->kp[i], P->C[i], P->n[i] / 64, P->m[i], P->k[i],
                                         P->n[i], s);
        if (st != BMM_OK) return st;
    }
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

}  // namespace

extern "C" {

bmm_status bmm_batched_plan_create(int32_t count, const int32_t* ops, const uint64_t* const* A,
                                   const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                                   const int64_t* k, const int64_t* n, bmm_batched_plan* plan) {
    return bmm_batched_plan_create_ex(count, ops, A, B, C, m, k, n, BMM_PATH_AUTO, plan);
}

bmm_status bmm_batched_plan_create_ex(int32_t count, const int32_t* ops,
                                      const uint64_t* const* A, const uint64_t* const* B,
                                      uint64_t* const* C, const int64_t* m, const int64_t* k,
                                      const int64_t* n, int32_t path, bmm_batched_plan* plan) {
    if (!plan) return BMM_ERR_INVALID;
    *plan = nullptr;
    if (path != BMM_PATH_AUTO && path != BMM_PATH_POPC && !is_tc_path(path))
        return path == BMM_PATH_TC_I8 ? BMM_ERR_UNSUPPORTED : BMM_ERR_INVALID;
    bmm_status st = check_batch(count, ops, A, B, C, m, k, n);
    if (st != BMM_OK) return st;
    if (path == BMM_PATH_AUTO) path = auto_path();
    if (is_tc_path(path) && !tc_path_available()) return BMM_ERR_UNSUPPORTED;
    bmm_batched_plan_s* P = new bmm_batched_plan_s();
    cudaGetDevice(&P->device);
    P->count = count;
    P->op.assign(ops, ops + count);
    P->A.assign(A, A + count);
    P->B.assign(B, B + count);
    P->C.assign(C, C + count);
    P->m.assign(m, m + count);
    P->k.assign(k, k + count);
    P->n.assign(n, n + count);
    st = plan_build(P, path);
    if (st != BMM_OK) {
        if (P->dmem) cudaFree(P->dmem);
        delete P;
        return st;
    }
    *plan = P;
    return BMM_OK;
}

bmm_status bmm_batched_plan_run(bmm_batched_plan plan, bmm_stream_t stream) {
    if (!plan) return BMM_ERR_INVALID;
    return plan_run(plan, (cudaStream_t)stream);
}

bmm_status bmm_batched_plan_path(bmm_batched_plan plan, int32_t* path) {
    if (!plan || !path) return BMM_ERR_INVALID;
    *path = !plan->tc     ? BMM_PATH_POPC
            : plan->fp4  ? BMM_PATH_TC_FP4_PAIR
            : plan->pair ? BMM_PATH_TC_FP8_PAIR
                         : BMM_PATH_TC_FP8;
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
