// lbm_batch.cu -- the batch entry points of the C ABI (include/lbm.h): many independent cases
// advanced together, CUDA graph replay of their steps, and the tuner.
//
// A step of the batch is a set of work items, each on a fixed branch stream:
//  * a group launch (batch_kernels.cu): all cases of one grid size, tile shape and kernel
//    variant in one grid, blockIdx.y = case;
//  * a dedicated launch: the single-case step kernel for one case.
// Items of different branches run concurrently; an item's successive steps stay on its branch,
// so stream order alone carries each case's dependence on its previous step and a graph of K
// steps needs one fork at its start and one join at its end, no barrier between steps.
// The tuner picks, per size class, the tile shape of the group launch or dedicated launches,
// whichever ran faster on this GPU, and the storage of cases that leave it open.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_ctx.h"
#include "lbm_internal.h"
#include "storage.cuh"

namespace {
constexpr int kBranches = 8;  // concurrent branch streams
}

struct BatchItem {
    int group;       // index into groups, or -1
    int dedicated;   // case index of a dedicated launch, or -1
    long long cells;
    int branch;
};

struct lbm_batch {
    int lattice;
    int device;
    cudaStream_t stream;
    bool own_stream;
    cudaStream_t branch[kBranches];
    cudaEvent_t fork_ev;
    cudaEvent_t join_ev[kBranches];
    std::vector<lbm_ctx*> cases;
    std::vector<int> tx_shift, ty_shift;  // tile shape per case (log2 extents in x and y)
    std::vector<char> dedicated;          // 1: the case runs the single-case kernel on its own
    std::vector<char> auto_storage;       // 1 where the case left its storage to the tuner
    std::vector<int> table_cur;           // each case's current buffer when the plan was built
    std::vector<long long> table_version; // each case's version when the plan was built
    std::vector<lbm::BatchLaunch> groups;
    std::vector<BatchItem> items;
    bool plan_valid;
    int flip;                             // steps since the plan was built, mod 2
    int graph_steps;
    cudaGraphExec_t graph_exec[2];
    long long launches;
    long long cells;
    char err[512];
};

namespace {

thread_local char g_batch_error[512] = "no error";

int berr(lbm_batch* b, int code, const char* fmt, ...) {
    char* dst = b ? b->err : g_batch_error;
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    // a failed allocation is reported here, synchronously, and is not sticky: clear it, or the
    // next launch's error check would report it again
    if (code == LBM_ENOMEM) (void)cudaGetLastError();
    return code;
}

#define LBM_BCUDA(b, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return berr((b), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,          \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

void drop_batch_graphs(lbm_batch* b) {
    for (int k = 0; k < 2; ++k)
        if (b->graph_exec[k]) {
            cudaGraphExecDestroy(b->graph_exec[k]);
            b->graph_exec[k] = nullptr;
        }
}

void free_batch(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < kBranches; ++k)
        if (b->branch[k]) cudaStreamSynchronize(b->branch[k]);
    drop_batch_graphs(b);
    for (lbm_ctx* c : b->cases) {
        if (!c) continue;
        c->batch_owned = false;
        lbm_destroy(c);
    }
    for (int k = 0; k < kBranches; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int next_pow2_shift(int n) {
    int s = 0;
    while ((1 << s) < n) ++s;
    return s;
}

long long case_cells(const lbm_ctx* c) { return c->P.N; }

// The bytes of every parameter a group launch takes from its first case for all of its cases
// (batch_step_kernel): the grid, walls, kernel variant and storage, the propagation and flux
// weights, the phase-field relaxation and interface constants and the storage shifts. Cases with
// equal keys differ only in their fluid properties (tau_f, density and viscosity ratio, surface
// tension, body force), which the kernel reads per case.
std::string group_key(const lbm::Params& P, int tx_shift, int ty_shift) {
    std::string k;
    auto put = [&](const void* v, size_t n) { k.append(static_cast<const char*>(v), n); };
    const int ints[] = {P.Q, P.nx, P.ny, P.nz, P.general, P.storage, P.walls, P.phi_ref_fx, tx_shift, ty_shift};
    const float floats[] = {P.lw_m, P.lw_p, P.flux_as, P.flux_bs, P.tau_phi, P.omega_g, P.grad_s, P.grad_k,
                            P.rho2, P.four_over_delta, P.w0, P.phi_ref};
    put(ints, sizeof ints);
    put(floats, sizeof floats);
    return k;
}

// Group launches for the cases in `which` (dedicated cases excluded by the caller): cases with
// equal group keys (one grid size, tile shape, kernel variant, storage and shared parameters),
// up to kMaxLaunchCases per launch.
void build_groups(const lbm_batch* b, const std::vector<int>& which, std::vector<lbm::BatchLaunch>& groups,
                  std::vector<long long>* group_cells) {
    groups.clear();
    if (group_cells) group_cells->clear();
    std::map<std::string, std::vector<int>> by_class;
    for (int k : which) by_class[group_key(b->cases[k]->P, b->tx_shift[k], b->ty_shift[k])].push_back(k);
    for (auto& kv : by_class) {
        const std::vector<int>& ks = kv.second;
        for (size_t i = 0; i < ks.size(); i += lbm::kMaxLaunchCases) {
            groups.emplace_back();
            lbm::BatchLaunch& L = groups.back();
            std::memset(&L, 0, sizeof(L));
            const int n = (int)std::min<size_t>(lbm::kMaxLaunchCases, ks.size() - i);
            const lbm::Params& P0 = b->cases[ks[i]]->P;
            L.n_cases = n;
            L.tx_shift = b->tx_shift[ks[i]];
            L.ty_shift = b->ty_shift[ks[i]];
            const int tx = 1 << L.tx_shift, ty = 1 << L.ty_shift;
            const int tz = lbm::kBatchThreads >> (L.tx_shift + L.ty_shift);
            L.ntx = (P0.nx + tx - 1) / tx;
            L.nty = (P0.ny + ty - 1) / ty;
            L.ntz = (P0.nz + tz - 1) / tz;
            L.general = P0.general;
            L.storage = P0.storage;
            long long cells = 0;
            for (int j = 0; j < n; ++j) {
                const lbm_ctx* c = b->cases[ks[i + j]];
                L.cases[j].P = c->P;
                L.cases[j].fg[0] = c->fg[0];
                L.cases[j].fg[1] = c->fg[1];
                L.cases[j].cur = c->cur;
                cells += case_cells(c);
            }
            if (group_cells) group_cells->push_back(cells);
        }
    }
}

// Work items of the cases in `which` and their branches: the largest first, each to the branch
// with the fewest cells so far.
void build_items(const lbm_batch* b, const std::vector<int>& which, std::vector<lbm::BatchLaunch>& groups,
                 std::vector<BatchItem>& items) {
    std::vector<int> grouped;
    items.clear();
    for (int k : which) {
        if (b->dedicated[k]) items.push_back(BatchItem{-1, k, case_cells(b->cases[k]), 0});
        else grouped.push_back(k);
    }
    std::vector<long long> gcells;
    build_groups(b, grouped, groups, &gcells);
    for (size_t g = 0; g < groups.size(); ++g) items.push_back(BatchItem{(int)g, -1, gcells[g], 0});
    std::sort(items.begin(), items.end(), [](const BatchItem& a, const BatchItem& c) { return a.cells > c.cells; });
    long long load[kBranches] = {0};
    for (BatchItem& it : items) {
        int best = 0;
        for (int r = 1; r < kBranches; ++r)
            if (load[r] < load[best]) best = r;
        it.branch = best;
        load[best] += it.cells;
    }
}

// One step of every item, each on its branch, at step parity `flip`.
int launch_items(lbm_batch* b, std::vector<lbm::BatchLaunch>& groups, const std::vector<BatchItem>& items, int flip,
                 long long* launches) {
    for (const BatchItem& it : items) {
        cudaStream_t s = b->branch[it.branch];
        if (it.group >= 0) {
            lbm::BatchLaunch& L = groups[it.group];
            L.flip = flip;
            LBM_BCUDA(b, lbm::launch_batch_group(b->lattice, L, s));
            *launches += 1;
        } else {
            lbm_ctx* c = b->cases[it.dedicated];
            const int par = b->table_cur[it.dedicated] ^ flip;
            int n = 0;
            LBM_BCUDA(b, lbm::launch_step(c->P, lbm::SCHEME_DF, c->fg[par], c->fg[1 - par], nullptr, s, &n));
            *launches += n;
        }
    }
    return LBM_OK;
}

int fork_branches(lbm_batch* b) {
    LBM_BCUDA(b, cudaEventRecord(b->fork_ev, b->stream));
    for (int r = 0; r < kBranches; ++r) LBM_BCUDA(b, cudaStreamWaitEvent(b->branch[r], b->fork_ev, 0));
    return LBM_OK;
}

int join_branches(lbm_batch* b) {
    for (int r = 0; r < kBranches; ++r) {
        LBM_BCUDA(b, cudaEventRecord(b->join_ev[r], b->branch[r]));
        LBM_BCUDA(b, cudaStreamWaitEvent(b->stream, b->join_ev[r], 0));
    }
    return LBM_OK;
}

// n steps of the items from parity flip0 between a fork and a join on the batch stream. With
// alternate = false every launch uses flip0 (the tuner's trials: read the current state, write
// the other buffer, never the state itself).
int run_steps(lbm_batch* b, std::vector<lbm::BatchLaunch>& groups, const std::vector<BatchItem>& items, int n,
              int flip0, long long* launches, bool alternate = true) {
    int rc = fork_branches(b);
    if (rc) return rc;
    int flip = flip0;
    for (int k = 0; k < n && rc == LBM_OK; ++k) {
        rc = launch_items(b, groups, items, flip, launches);
        if (alternate) flip ^= 1;
    }
    int rc2 = join_branches(b);
    return rc ? rc : rc2;
}

void snapshot(lbm_batch* b) {
    const size_t n = b->cases.size();
    b->table_cur.assign(n, 0);
    b->table_version.assign(n, 0);
    for (size_t k = 0; k < n; ++k) {
        b->table_cur[k] = b->cases[k]->cur;
        b->table_version[k] = b->cases[k]->version;
    }
}

// Rebuilds the plan when a case changed outside the batch (its own lbm_step, lbm_init_phi,
// lbm_set_pops) or the tuner changed it.
int refresh(lbm_batch* b) {
    bool stale = !b->plan_valid;
    for (size_t k = 0; k < b->cases.size() && !stale; ++k) {
        const lbm_ctx* c = b->cases[k];
        if (c->cur != (b->table_cur[k] ^ b->flip) || c->version != b->table_version[k]) stale = true;
    }
    if (!stale) return LBM_OK;
    drop_batch_graphs(b);
    b->flip = 0;
    snapshot(b);
    std::vector<int> all(b->cases.size());
    for (size_t k = 0; k < all.size(); ++k) all[k] = (int)k;
    build_items(b, all, b->groups, b->items);
    b->plan_valid = true;
    return LBM_OK;
}

int capture_batch_graph(lbm_batch* b, int start_flip) {
    cudaGraph_t graph = nullptr;
    LBM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    long long launches = 0;
    int rc = run_steps(b, b->groups, b->items, b->graph_steps, start_flip, &launches);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc == LBM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec[start_flip], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    if (e != cudaSuccess) {
        b->graph_exec[start_flip] = nullptr;
        return berr(b, LBM_ECUDA, "capturing the batch step graph failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

int check_batch(lbm_batch* b) {
    if (!b) return berr(nullptr, LBM_EINVAL, "null batch");
    LBM_BCUDA(b, cudaSetDevice(b->device));
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_batch_default_opts(lbm_batch_opts* o) {
    if (!o) return;
    o->stream = nullptr;
    o->graph_steps = 32;
}

int lbm_batch_create(lbm_batch** out, int n_cases, const lbm_case* cases, const lbm_batch_opts* opts) {
    if (!out) return berr(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_cases < 1 || !cases) return berr(nullptr, LBM_EINVAL, "need n_cases >= 1 and a case array");
    lbm_batch_opts o;
    lbm_batch_default_opts(&o);
    if (opts) o = *opts;
    if (o.graph_steps < 0 || o.graph_steps == 1 || (o.graph_steps & 1))
        return berr(nullptr, LBM_EINVAL, "graph_steps must be 0 or an even count >= 2 (got %d)", o.graph_steps);
    const int lattice = cases[0].lattice;
    long long total = 0;
    for (int k = 0; k < n_cases; ++k) {
        const lbm_case& cs = cases[k];
        if (cs.lattice != lattice)
            return berr(nullptr, LBM_EINVAL, "case %d: every case of a batch needs the same lattice", k);
        if (cs.storage < 0 || cs.storage > LBM_STORAGE_AUTO)
            return berr(nullptr, LBM_EINVAL, "case %d: storage must be 0..2 or LBM_STORAGE_AUTO (got %d)", k, cs.storage);
        if (cs.grid[0] < 3 || cs.grid[1] < 3 || cs.grid[2] < 1)
            return berr(nullptr, LBM_EINVAL, "case %d: grid too small", k);
        total += (long long)cs.grid[0] * cs.grid[1] * cs.grid[2];
    }
    if (total >= (1ll << 40)) return berr(nullptr, LBM_EINVAL, "the batch holds too many cells (%lld)", total);

    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return berr(nullptr, LBM_ENOMEM, "host allocation failed");
    std::snprintf(b->err, sizeof b->err, "no error");
    b->lattice = lattice;
    b->graph_steps = o.graph_steps;
    b->cells = total;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return berr(nullptr, LBM_ECUDA, "no CUDA device available");
    }
    auto fail = [&](int code) {
        std::snprintf(g_batch_error, sizeof g_batch_error, "%s", b->err);
        free_batch(b);
        return code;
    };
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(berr(b, LBM_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e)));
        b->own_stream = true;
    }
    {
        cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
        for (int r = 0; r < kBranches && e == cudaSuccess; ++r) {
            e = cudaStreamCreateWithFlags(&b->branch[r], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[r], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail(berr(b, LBM_ECUDA, "creating branch streams failed: %s", cudaGetErrorString(e)));
    }
    b->cases.assign(n_cases, nullptr);
    b->tx_shift.assign(n_cases, 0);
    b->ty_shift.assign(n_cases, 0);
    b->dedicated.assign(n_cases, 0);
    b->auto_storage.assign(n_cases, 0);
    for (int k = 0; k < n_cases; ++k) {
        const lbm_case& cs = cases[k];
        lbm_opts co;
        lbm_default_opts(&co);
        co.storage = (cs.storage == LBM_STORAGE_AUTO) ? LBM_STORAGE_FP32 : cs.storage;
        co.walls = cs.walls;
        if (cs.courant != 0) co.courant = cs.courant;
        co.stream = b->stream;
        co.graph_steps = 0;
        b->auto_storage[k] = cs.storage == LBM_STORAGE_AUTO;
        int rc = lbm::create_ctx(&b->cases[k], cs.grid, cs.lattice, cs.tau_f, cs.tau_g, cs.M, cs.xi, cs.sigma,
                                 cs.rho_ratio, cs.mu_ratio, cs.body_force, &co, LBM_STORAGE_FP32);
        if (rc) return fail(berr(b, rc, "case %d: %s", k, lbm_last_error(nullptr)));
        b->cases[k]->batch_owned = true;
        // Default form, the choice the tuner made for most classes on GB300: a case whose rows
        // fill whole warps (nx a multiple of 32, at least 2^15 cells) runs in dedicated launches;
        // the others in group launches whose tile is 2^a cells wide, 2^a the largest power of two
        // up to 32 that divides nx (at least 8), then 8 in y (2D: all the rest), then z.
        const lbm::Params& P = b->cases[k]->P;
        b->dedicated[k] = (P.nx % 32 == 0 && P.N >= 32768) ? 1 : 0;
        int txs = 3;
        while (txs < 5 && P.nx % (1 << (txs + 1)) == 0) ++txs;
        if (txs > next_pow2_shift(P.nx)) txs = next_pow2_shift(P.nx);
        int tys = (P.nz == 1) ? 7 - txs : (7 - txs < 3 ? 7 - txs : 3);
        if (P.nz > 1 && tys > next_pow2_shift(P.ny)) tys = next_pow2_shift(P.ny);
        b->tx_shift[k] = txs;
        b->ty_shift[k] = tys;
    }
    *out = b;
    return LBM_OK;
}

lbm_ctx* lbm_batch_case(lbm_batch* b, int k) {
    if (!b || k < 0 || k >= (int)b->cases.size()) return nullptr;
    return b->cases[k];
}

int lbm_batch_case_config(const lbm_batch* b, int k, int tile[3], int* storage, int* dedicated) {
    if (!b || k < 0 || k >= (int)b->cases.size()) return LBM_EINVAL;
    if (tile) {
        tile[0] = 1 << b->tx_shift[k];
        tile[1] = 1 << b->ty_shift[k];
        tile[2] = lbm::kBatchThreads >> (b->tx_shift[k] + b->ty_shift[k]);
    }
    if (storage) *storage = b->cases[k]->P.storage;
    if (dedicated) *dedicated = b->dedicated[k];
    return LBM_OK;
}

int lbm_batch_set_config(lbm_batch* b, int k, const int tile[3], int dedicated) {
    if (!b) return berr(nullptr, LBM_EINVAL, "null batch");
    if (k < 0 || k >= (int)b->cases.size()) return berr(b, LBM_EINVAL, "no case %d", k);
    if (tile) {
        const int tx = tile[0], ty = tile[1], tz = tile[2];
        const bool pow2 = tx > 0 && ty > 0 && tz > 0 && !(tx & (tx - 1)) && !(ty & (ty - 1)) && !(tz & (tz - 1));
        if (!pow2 || tx * ty * tz != lbm::kBatchThreads || (b->cases[k]->P.nz == 1 && tz != 1))
            return berr(b, LBM_EINVAL, "tile must be powers of two with %d cells (tz = 1 in 2D)", lbm::kBatchThreads);
        b->tx_shift[k] = next_pow2_shift(tx);
        b->ty_shift[k] = next_pow2_shift(ty);
    }
    b->dedicated[k] = dedicated ? 1 : 0;
    b->plan_valid = false;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int trial_steps) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (trial_steps < 1) return berr(b, LBM_EINVAL, "trial_steps must be >= 1 (got %d)", trial_steps);
    const int n = (int)b->cases.size();
    std::map<std::tuple<int, int, int>, std::vector<int>> classes;  // size classes
    for (int k = 0; k < n; ++k) {
        const lbm::Params& P = b->cases[k]->P;
        classes[std::make_tuple(P.nx, P.ny, P.nz)].push_back(k);
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    LBM_BCUDA(b, cudaEventCreate(&ev0));
    LBM_BCUDA(b, cudaEventCreate(&ev1));
    struct EventGuard {
        cudaEvent_t a, c;
        ~EventGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(c);
        }
    } guard{ev0, ev1};
    drop_batch_graphs(b);
    snapshot(b);  // trial launches read each case's current buffer (flip 0) and write the other
    std::vector<lbm::BatchLaunch> groups;
    std::vector<BatchItem> items;
    for (auto& kv : classes) {
        const std::vector<int>& members = kv.second;
        const lbm::Params& P0 = b->cases[members[0]]->P;
        // storage is open where every member that asks for it holds no state yet
        bool open = false;
        for (int k : members)
            if (b->auto_storage[k] && !b->cases[k]->initialised) open = true;
        const std::vector<int> storages = open ? std::vector<int>{0, 1, 2} : std::vector<int>{-1};
        // modes: a group launch per tile shape 2^a x 2^b x 2^c = 128 (a >= 3, no extent beyond the
        // grid's next power of two), and dedicated launches (shape (-1, -1))
        const int sx = next_pow2_shift(P0.nx), sy = next_pow2_shift(P0.ny), sz = next_pow2_shift(P0.nz);
        std::vector<std::pair<int, int>> modes;
        for (int a = 3; a <= 7; ++a)
            for (int c2 = 0; c2 <= 7 - a; ++c2) {
                const int zc = 7 - a - c2;
                if (a > sx || c2 > sy || zc > sz || (P0.nz == 1 && zc != 0)) continue;
                modes.emplace_back(a, c2);
            }
        if (modes.empty()) modes.emplace_back(b->tx_shift[members[0]], b->ty_shift[members[0]]);
        modes.emplace_back(-1, -1);
        float best = -1.f;
        int best_s = -1;
        std::pair<int, int> best_m = modes[0];
        for (int s : storages) {
            if (s >= 0)
                for (int k : members) {
                    if (!b->auto_storage[k] || b->cases[k]->initialised) continue;
                    rc = lbm::set_ctx_storage(b->cases[k], s);
                    if (rc) return berr(b, rc, "case %d: %s", k, b->cases[k]->err);
                }
            for (int k : members)
                if (!b->cases[k]->initialised)
                    LBM_BCUDA(b, lbm::launch_fill_rest(b->cases[k]->P, b->cases[k]->fg[b->cases[k]->cur], b->stream));
            for (const auto& m : modes) {
                for (int k : members) {
                    b->dedicated[k] = m.first < 0;
                    if (m.first >= 0) {
                        b->tx_shift[k] = m.first;
                        b->ty_shift[k] = m.second;
                    }
                }
                build_items(b, members, groups, items);
                long long launches = 0;
                rc = run_steps(b, groups, items, 1, 0, &launches, false);  // warm-up
                if (rc) return rc;
                LBM_BCUDA(b, cudaEventRecord(ev0, b->stream));
                rc = run_steps(b, groups, items, trial_steps, 0, &launches, false);
                if (rc) return rc;
                LBM_BCUDA(b, cudaEventRecord(ev1, b->stream));
                LBM_BCUDA(b, cudaEventSynchronize(ev1));
                float ms = 0.f;
                LBM_BCUDA(b, cudaEventElapsedTime(&ms, ev0, ev1));
                b->launches += launches;
                if (best < 0.f || ms < best) {
                    best = ms;
                    best_s = s;
                    best_m = m;
                }
            }
        }
        for (int k : members) {
            b->dedicated[k] = best_m.first < 0;
            if (best_m.first >= 0) {
                b->tx_shift[k] = best_m.first;
                b->ty_shift[k] = best_m.second;
            }
            if (best_s >= 0 && b->auto_storage[k] && !b->cases[k]->initialised) {
                rc = lbm::set_ctx_storage(b->cases[k], best_s);
                if (rc) return berr(b, rc, "case %d: %s", k, b->cases[k]->err);
            }
        }
    }
    b->plan_valid = false;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (n < 0) return berr(b, LBM_EINVAL, "n must be >= 0 (got %d)", n);
    for (size_t k = 0; k < b->cases.size(); ++k)
        if (!b->cases[k]->initialised)
            return berr(b, LBM_ESTATE, "case %zu has no state: call lbm_init_phi on lbm_batch_case(b, %zu)", k, k);
    rc = refresh(b);
    if (rc) return rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LBM_BCUDA(b, cudaStreamIsCapturing(b->stream, &cap));
    if (b->graph_steps > 0 && cap == cudaStreamCaptureStatusNone) {
        const long long per_graph = (long long)b->items.size();  // one launch per item and step
        while (n >= b->graph_steps) {
            if (!b->graph_exec[b->flip]) {
                rc = capture_batch_graph(b, b->flip);
                if (rc) return rc;
            }
            LBM_BCUDA(b, cudaGraphLaunch(b->graph_exec[b->flip], b->stream));
            b->launches += per_graph * b->graph_steps;
            n -= b->graph_steps;  // an even count leaves flip unchanged
        }
    }
    if (n > 0) {
        long long launches = 0;
        rc = run_steps(b, b->groups, b->items, n, b->flip, &launches);
        if (rc) return rc;
        b->launches += launches;
        b->flip ^= (n & 1);
    }
    for (size_t k = 0; k < b->cases.size(); ++k) b->cases[k]->cur = b->table_cur[k] ^ b->flip;
    return LBM_OK;
}

long long lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

long long lbm_batch_cells(const lbm_batch* b) { return b ? b->cells : 0; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_batch_error; }

void lbm_batch_destroy(lbm_batch* b) { free_batch(b); }

}  // extern "C"
