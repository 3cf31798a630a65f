// Batched ensemble: the C ABI (sca_batch_*) and its host side: the plan that packs lattices
// into cluster units for the persistent cluster engine (sca_batch.cu), the streaming engine's
// classes of equal size and rule (sca_wave_batch.cu), captured runs, and the shape tuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>
#include <string>
#include <vector>

#include "sca.h"
#include "sca_batch.h"

namespace sca {
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);
int make_rule(const sca_params &prm, Rule &R);

constexpr uint32_t kBatchMaxL = 2048;          // observation teams span at most one warp
constexpr int kBatchMaxObs = 64;
constexpr size_t kBatchSmemCap = 200 * 1024;   // default shared memory per CTA for one part

// Fewest CTAs whose shared memory holds the lattice (parts may differ by one row); among
// those, prefer a count that divides the cluster so units have no idle CTAs.
static uint32_t parts_needed(uint32_t L, int C, size_t cap)
{
    uint32_t g0 = 0;
    for (uint32_t G = 1; G <= (uint32_t)C; ++G)
        if (batch_part_smem(L, G) <= cap && (L / G) >= 2) { g0 = G; break; }
    if (g0 == 0) return 0;
    for (uint32_t G = g0; G <= (uint32_t)C; ++G)
        if (C % G == 0) return G;
    return g0;
}
}  // namespace sca

using namespace sca;

struct sca_batch {
    std::vector<sca_params> P;
    std::vector<BatchLattice> lat;     // host copy; G, part_off depend on the plan
    std::vector<uint64_t> state_off;
    uint32_t count = 0;
    size_t state_words = 0;
    uint32_t *state = nullptr;         // all lattices' canonical words
    BatchLattice *lat_d = nullptr;
    BatchSlot *slots_d = nullptr;
    int n_units = 0;
    uint32_t *counter = nullptr;
    uint64_t *times_d = nullptr;
    uint64_t *unit_ns = nullptr;       // 2 per unit (capacity: one unit per lattice)
    std::vector<int32_t> unit_first;   // first lattice of each unit (host copy)
    ObsPartial *part = nullptr;
    size_t part_cap = 0;               // partial entries available
    ObsDev *res = nullptr;             // count x kBatchMaxObs
    ObsDev *res_h = nullptr;           // pinned copy
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t t = 0;
    int C = 8, threads = 512, clusters = 0;
    size_t smem = 0, cap = 0;
    // streaming engine: lattices grouped by (size, rule) into classes, each run as its own
    // chain of launches on its own stream
    int engine = 0;                    // requested: 0 automatic, 1 clusters, 2 streaming
    uint32_t *state2 = nullptr;        // second state buffer (ping-pong)
    struct WBClass {
        uint32_t L = 0, n_lat = 0, rows = 0, n_items = 0;
        Rule R{};
        WBItem *items = nullptr;       // device
        uint64_t *off = nullptr;       // device: members' state offsets
        uint32_t *dst = nullptr;       // device: members' lattice indices
        void *chunks = nullptr;        // device: observation scratch
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<WBClass> classes;
    cudaEvent_t fork = nullptr;
    bool wb_ready = false;
    // captured run (reused while the observation times and start time repeat)
    cudaGraphExec_t graph = nullptr;
    std::vector<uint64_t> graph_times;
    uint64_t graph_t0 = ~0ull;
};

static void batch_drop_graph(sca_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_times.clear();
    b->graph_t0 = ~0ull;
}

// Pack lattices into cluster units: lattices of equal (L, G, rule cost) share units of C/G
// lattices; units are ordered by decreasing estimated work so the dynamic queue balances.
static int batch_plan(sca_batch *b, int C, int threads, size_t cap = kBatchSmemCap)
{
    const uint32_t n = b->count;
    std::vector<uint32_t> G(n);
    size_t smem = 0;
    for (uint32_t i = 0; i < n; ++i) {
        G[i] = parts_needed(b->lat[i].L, C, cap);
        if (G[i] == 0) return fail(SCA_EINVAL, "lattice too large for the batch cluster size");
        smem = std::max(smem, batch_part_smem(b->lat[i].L, G[i]));
    }
    auto cost = [&](uint32_t i) {
        const Rule &R = b->lat[i].R;
        const double f = R.mode == 0 ? 1.0 : R.mode == 1 ? 1.0 + 1.5 * R.n_draws : 24.0;
        return (double)b->lat[i].L * b->lat[i].L / G[i] * f;
    };
    // groups of interchangeable lattices: same parts, same size, same rule cost
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    auto key = [&](uint32_t i) { return std::make_tuple(G[i], b->lat[i].L, cost(i)); };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return key(x) > key(y); });
    struct Unit { double cost; std::vector<BatchSlot> s; };
    std::vector<Unit> units;
    for (size_t i = 0; i < order.size();) {
        const uint32_t g = G[order[i]];
        const uint32_t per = (uint32_t)C / g;
        Unit u;
        u.cost = cost(order[i]);
        u.s.assign(C, BatchSlot{-1, 0, (int16_t)g});
        const auto k0 = key(order[i]);
        for (uint32_t k = 0; k < per && i < order.size() && key(order[i]) == k0; ++k, ++i)
            for (uint32_t p = 0; p < g; ++p) u.s[k * g + p] = BatchSlot{(int32_t)order[i], (int16_t)p, (int16_t)g};
        units.push_back(u);
    }
    std::stable_sort(units.begin(), units.end(), [](const Unit &x, const Unit &y) { return x.cost > y.cost; });
    std::vector<BatchSlot> slots;
    b->unit_first.clear();
    for (auto &u : units) {
        slots.insert(slots.end(), u.s.begin(), u.s.end());
        b->unit_first.push_back(u.s[0].lattice);
    }
    uint32_t part_off = 0;
    for (uint32_t k = 0; k < n; ++k) {
        b->lat[k].G = G[k];
        b->lat[k].part_off = part_off;
        part_off += G[k] * kBatchMaxObs;
    }
    int max_clusters = 0;
    cudaError_t e = batch_max_clusters(C, threads, smem, &max_clusters);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // a refused shape must not surface at a later launch check
        return cuda_fail(e, "cudaOccupancyMaxActiveClusters");
    }
    if (max_clusters < 1) return fail(SCA_EINVAL, "batch launch shape does not fit the GPU");
    // device tables
    if (b->slots_d) cudaFree(b->slots_d);
    b->slots_d = nullptr;
    e = cudaMalloc(&b->slots_d, slots.size() * sizeof(BatchSlot));
    if (e != cudaSuccess) return fail(SCA_ENOMEM, "batch slot table");
    e = cudaMemcpyAsync(b->slots_d, slots.data(), slots.size() * sizeof(BatchSlot),
                        cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->lat_d, b->lat.data(), n * sizeof(BatchLattice), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch tables");
    b->n_units = (int)units.size();
    b->cap = cap;
    b->C = C;
    b->threads = threads;
    b->smem = smem;
    b->clusters = std::min(max_clusters, b->n_units);
    batch_drop_graph(b);
    return SCA_OK;
}

extern "C" {

int sca_batch_reset(sca_batch *b)
{
    if (!b) return fail(SCA_EINVAL, "NULL batch");
    for (uint32_t i = 0; i < b->count; ++i) {
        const size_t bytes = (size_t)b->lat[i].L * b->lat[i].L / 4;
        char *p = (char *)(b->state + b->state_off[i]);
        cudaError_t e = cudaMemsetAsync(p, 0x00, bytes / 2, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(p + bytes / 2, 0xFF, bytes / 2, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    b->t = 0;
    return SCA_OK;
}

void sca_batch_free(sca_batch *b);

int sca_batch_init(const sca_params *params, uint32_t count, void *stream, sca_batch **out)
{
    if (!params || !out || count == 0) return fail(SCA_EINVAL, "NULL argument or empty batch");
    *out = nullptr;
    sca_batch *b = new sca_batch();
    b->count = count;
    b->P.assign(params, params + count);
    b->lat.resize(count);
    b->state_off.resize(count);
    size_t words = 0;
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t L = params[i].L;
        if (L < 128 || L % 64 != 0 || L > kBatchMaxL) {
            delete b;
            return fail(SCA_EINVAL, "batch lattices need L a multiple of 64 in [128, 2048]");
        }
        if (params[i].Ly != 0 && params[i].Ly != L) {
            delete b;
            return fail(SCA_EINVAL, "batch lattices are square (Ly = 0 or L)");
        }
        if (params[i].dynamics != SCA_DYN_SCA) {
            delete b;
            return fail(SCA_EINVAL, "batch lattices run the SCA dynamics");
        }
        BatchLattice &lt = b->lat[i];
        std::memset(&lt, 0, sizeof(lt));
        int rc = make_rule(params[i], lt.R);
        if (rc) { delete b; return rc; }
        lt.L = L;
        lt.W = L / 64;
        lt.V = (lt.W % 4 == 0) ? 4 : (lt.W % 2 == 0) ? 2 : 1;
        lt.state_off = words;
        b->state_off[i] = words;
        words += (size_t)L * L / 16;
        words = (words + 63) & ~(size_t)63;          // 256-byte alignment per lattice
    }
    b->state_words = words;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    b->part_cap = 0;
    for (uint32_t i = 0; i < count; ++i) b->part_cap += 8 * (size_t)kBatchMaxObs;   // G <= 8
    cudaError_t e = cudaMalloc(&b->state, words * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->lat_d, count * sizeof(BatchLattice));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->times_d, kBatchMaxObs * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->unit_ns, 2 * (size_t)count * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->part, b->part_cap * sizeof(ObsPartial));
    if (e == cudaSuccess) e = cudaMalloc(&b->res, (size_t)count * kBatchMaxObs * sizeof(ObsDev));
    if (e == cudaSuccess) e = cudaMallocHost(&b->res_h, (size_t)count * kBatchMaxObs * sizeof(ObsDev));
    if (e != cudaSuccess) {
        sca_batch_free(b);
        return fail(SCA_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    int rc = sca_batch_reset(b);
    if (!rc) rc = batch_plan(b, 8, 512);
    if (rc) { sca_batch_free(b); return rc; }
    *out = b;
    return SCA_OK;
}

int sca_batch_set_shape(sca_batch *b, int cluster, int threads)
{
    if (!b) return fail(SCA_EINVAL, "NULL batch");
    if (!((cluster >= 1 && cluster <= 8) || cluster == 16) ||
        !(threads == 128 || threads == 256 || threads == 384 || threads == 512))
        return fail(SCA_EINVAL, "cluster must be 1..8 or 16 and threads 128..512");
    return batch_plan(b, cluster, threads);
}

int sca_batch_get_shape(const sca_batch *b, int *cluster, int *threads, int *clusters_launched,
                        int *units)
{
    if (!b) return fail(SCA_EINVAL, "NULL batch");
    if (cluster) *cluster = b->C;
    if (threads) *threads = b->threads;
    if (clusters_launched) *clusters_launched = b->clusters;
    if (units) *units = b->n_units;
    return SCA_OK;
}

// ------------------------------------------------------------------ streaming engine (host)
static bool same_rule(const Rule &a, const Rule &c)
{
    return a.mode == c.mode && a.n_draws == c.n_draws && a.np == c.np && a.nq == c.nq && a.Pp == c.Pp &&
           a.Pq == c.Pq && a.Tp == c.Tp && a.Tq == c.Tq;
}

static bool wb_supported(const sca_batch *b)
{
    for (uint32_t i = 0; i < b->count; ++i)
        if (!wave_batch_supported(b->lat[i].L, b->lat[i].R)) return false;
    return true;
}

static void wb_free(sca_batch *b)
{
    for (auto &c : b->classes) {
        cudaFree(c.items);
        cudaFree(c.off);
        cudaFree(c.dst);
        cudaFree(c.chunks);
        if (c.done) cudaEventDestroy(c.done);
    }
    // streams are shared between classes: destroy each once
    std::vector<cudaStream_t> seen;
    for (auto &c : b->classes)
        if (c.st && std::find(seen.begin(), seen.end(), c.st) == seen.end()) seen.push_back(c.st);
    for (cudaStream_t s : seen) cudaStreamDestroy(s);
    b->classes.clear();
    if (b->fork) cudaEventDestroy(b->fork);
    b->fork = nullptr;
    cudaFree(b->state2);
    b->state2 = nullptr;
    b->wb_ready = false;
}

// Classes of equal (L, rule); bands of at most 512 rows (an even count, equal within a class);
// one work item per (lattice, band).
static int wb_setup(sca_batch *b)
{
    if (b->wb_ready) return SCA_OK;
    std::vector<int> cls(b->count, -1);
    std::vector<std::vector<uint32_t>> members;
    std::vector<sca_batch::WBClass> classes;
    for (uint32_t i = 0; i < b->count; ++i) {
        int c = -1;
        for (size_t k = 0; k < classes.size(); ++k)
            if (classes[k].L == b->lat[i].L && same_rule(classes[k].R, b->lat[i].R)) { c = (int)k; break; }
        if (c < 0) {
            sca_batch::WBClass nc;
            nc.L = b->lat[i].L;
            nc.R = b->lat[i].R;
            classes.push_back(nc);
            members.emplace_back();
            c = (int)classes.size() - 1;
        }
        members[c].push_back(i);
    }
    b->classes = classes;
    cudaError_t e = cudaMalloc(&b->state2, b->state_words * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    const int n_streams = (int)std::min<size_t>(16, classes.size());
    std::vector<cudaStream_t> streams(n_streams, nullptr);
    for (int s = 0; s < n_streams && e == cudaSuccess; ++s)
        e = cudaStreamCreateWithFlags(&streams[s], cudaStreamNonBlocking);
    for (size_t k = 0; k < b->classes.size() && e == cudaSuccess; ++k) {
        auto &c = b->classes[k];
        c.st = streams[k % n_streams];
        c.n_lat = (uint32_t)members[k].size();
        // bands: enough work items for about one wave of warps per launch (a class's launches
        // form a chain, so a launch must not be a long sweep of few warps), but bands of at
        // least 4K + 8 rows (rounded to a power of two) so the recomputed halo stays moderate
        const uint32_t kmax = (uint32_t)wave_batch_max_k(c.R);
        uint32_t min_rows = 1;
        while (min_rows < 4 * kmax + 8) min_rows *= 2;
        const uint32_t V = (c.R.mode == 1 && (c.L / 64) % 4 == 0) ? 4u : 1u;
        const uint32_t groups_per_warp = 32u / ((c.L / 64) / V);
        const uint64_t want_items = (uint64_t)groups_per_warp * (uint64_t)sm_count() * 16u;
        uint32_t bands = 1;
        while ((uint64_t)c.n_lat * bands < want_items && c.L / (2 * bands) >= min_rows &&
               (c.L / (2 * bands)) % 2 == 0)
            bands *= 2;
        c.rows = c.L / bands;
        std::vector<WBItem> items;
        std::vector<uint64_t> off;
        std::vector<uint32_t> dst;
        for (uint32_t m : members[k]) {
            const uint64_t seed = b->P[m].seed;
            for (uint32_t q = 0; q < bands; ++q)
                items.push_back(WBItem{b->state_off[m], (uint32_t)seed, (uint32_t)(seed >> 32), q * c.rows, 0u});
            off.push_back(b->state_off[m]);
            dst.push_back(m);
        }
        c.n_items = (uint32_t)items.size();
        e = cudaMalloc(&c.items, items.size() * sizeof(WBItem));
        if (e == cudaSuccess) e = cudaMalloc(&c.off, off.size() * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc(&c.dst, dst.size() * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&c.chunks, obs_batch_scratch_bytes(c.n_lat, c.L));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaMemcpy(c.items, items.data(), items.size() * sizeof(WBItem), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.off, off.data(), off.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.dst, dst.data(), dst.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        // streams created so far belong to the classes (or to nobody if setup failed early)
        for (auto &c : b->classes) c.st = nullptr;
        for (cudaStream_t s : streams) if (s) cudaStreamDestroy(s);
        wb_free(b);
        return cuda_fail(e, "streaming batch setup");
    }
    b->wb_ready = true;
    return SCA_OK;
}

static bool use_streaming(const sca_batch *b)
{
    if (b->engine == 1) return false;
    return wb_supported(b);        // requested (2) or automatic (0): whenever every class fits
}

// Every class is an independent chain on its own stream: launches of up to K MCS between the
// observation times, the class's observation at each time, and a copy back into the first
// state buffer if the chain ended in the second.
static int wb_enqueue(sca_batch *b, uint32_t n)
{
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (auto &c : b->classes) {
        if (e != cudaSuccess) break;
        e = cudaStreamWaitEvent(c.st, b->fork, 0);
        uint64_t t = b->t;
        int cur = 0;
        uint32_t *buf[2] = {b->state, b->state2};
        const uint32_t kmax = (uint32_t)wave_batch_max_k(c.R);
        for (uint32_t ob = 0; ob < n && e == cudaSuccess; ++ob) {
            const uint64_t T = b->graph_times[ob];
            while (t < T && e == cudaSuccess) {
                uint32_t k = 1;
                while (2 * k <= kmax && 2 * k <= T - t) k *= 2;
                // a launch followed by one of the same k before the observation leaves it the
                // sx- planes but for the rows it starts its bands from
                const uint64_t rest = T - t - k;
                uint32_t k2 = 1;
                while (2 * k2 <= kmax && 2 * k2 <= rest) k2 *= 2;
                const bool sx_all = rest == 0 || k2 != k;
                e = launch_wave_batch(buf[cur], buf[cur ^ 1], c.items, c.n_items, c.L, c.rows, t, k, c.R, c.st,
                                      sx_all);
                cur ^= 1;
                t += k;
            }
            if (e == cudaSuccess)
                e = launch_observe_batch(buf[cur], c.off, c.n_lat, c.L, c.chunks, c.dst, n, b->res + ob, T, c.st);
        }
        if (e == cudaSuccess && cur == 1) e = launch_wave_batch_copy(b->state2, b->state, c.items, c.n_items, c.L, c.st);
        if (e == cudaSuccess) e = cudaEventRecord(c.done, c.st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c.done, 0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->res_h, b->res, (size_t)b->count * n * sizeof(ObsDev), cudaMemcpyDeviceToHost, b->stream);
    return e == cudaSuccess ? SCA_OK : cuda_fail(e, "streaming batch launch");
}

static int batch_enqueue(sca_batch *b, uint32_t n)
{
    if (use_streaming(b)) {
        int rc = wb_setup(b);
        if (rc) return rc;
        return wb_enqueue(b, n);
    }
    BatchArgs a;
    a.state = b->state;
    a.lat = b->lat_d;
    a.slots = b->slots_d;
    a.n_units = b->n_units;
    a.C = b->C;
    a.unit_counter = b->counter;
    a.times = b->times_d;
    a.n_times = (int)n;
    a.t0 = b->t;
    a.partials = b->part;
    a.unit_ns = b->unit_ns;
    cudaError_t e = cudaMemsetAsync(b->counter, 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = launch_batch(a, b->clusters, b->threads, b->smem, b->stream);
    if (e == cudaSuccess)
        e = launch_batch_finalize(b->lat_d, (int)b->count, b->part, b->times_d, (int)n, b->res, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->res_h, b->res, (size_t)b->count * n * sizeof(ObsDev),
                            cudaMemcpyDeviceToHost, b->stream);
    return e == cudaSuccess ? SCA_OK : cuda_fail(e, "batch launch");
}

int sca_batch_set_engine(sca_batch *b, int engine)
{
    if (!b || engine < 0 || engine > 2) return fail(SCA_EINVAL, "engine must be 0, 1 or 2");
    if (engine == 2 && !wb_supported(b))
        return fail(SCA_EINVAL, "the streaming engine needs L <= 2048 with a power-of-two row length "
                                "and dyadic or {0, 1} probabilities for every lattice");
    b->engine = engine;
    batch_drop_graph(b);
    return SCA_OK;
}

int sca_batch_get_engine(const sca_batch *b)
{
    if (!b) return fail(SCA_EINVAL, "NULL batch");
    return use_streaming(b) ? 2 : 1;
}

int sca_batch_run(sca_batch *b, const uint64_t *times, uint32_t n, sca_obs *out, double *ensemble_w2)
{
    if (!b || !times || n == 0) return fail(SCA_EINVAL, "NULL argument or no times");
    if (n > (uint32_t)kBatchMaxObs) return fail(SCA_EINVAL, "at most 64 observation times per run");
    uint64_t prev = b->t;
    for (uint32_t i = 0; i < n; ++i) {
        if (times[i] <= prev) return fail(SCA_EINVAL, "times must be increasing and after the current MCS");
        prev = times[i];
    }
    std::vector<uint64_t> tv(times, times + n);
    int rc = SCA_OK;
    if (!(b->graph && b->graph_t0 == b->t && b->graph_times == tv)) {
        batch_drop_graph(b);
        cudaError_t e = cudaMemcpyAsync(b->times_d, times, n * sizeof(uint64_t), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch times");
        cudaGraph_t g = nullptr;
        b->graph_times = tv;
        if (use_streaming(b)) {
            rc = wb_setup(b);                // allocations happen outside the capture
            if (rc) return rc;
        }
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        rc = batch_enqueue(b, n);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); b->graph_times.clear(); return rc; }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
        b->graph_times = tv;
        b->graph_t0 = b->t;
    }
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch run");
    b->t = times[n - 1];
    int first_bad = SCA_OK;
    for (uint32_t ob = 0; ob < n; ++ob) {
        double acc = 0.0;
        for (uint32_t i = 0; i < b->count; ++i) {
            sca_obs o;
            std::memcpy(&o, &b->res_h[(size_t)i * n + ob], sizeof(o));
            const double num = std::ldexp((double)o.num_hi, 64) + (double)o.num_lo;
            o.w2 = num / ((double)o.N * (double)o.N);
            if (o.status && !first_bad) first_bad = o.status;
            acc += o.w2;
            if (out) out[(size_t)i * n + ob] = o;
        }
        if (ensemble_w2) ensemble_w2[ob] = acc / b->count;
    }
    if (first_bad) return fail(first_bad, "a lattice's slopes do not close around the torus");
    return SCA_OK;
}

int sca_batch_get_state(sca_batch *b, uint32_t index, uint32_t *host_words, size_t n_words)
{
    if (!b || !host_words || index >= b->count) return fail(SCA_EINVAL, "bad argument");
    const size_t need = (size_t)b->lat[index].L * b->lat[index].L / 16;
    if (n_words < need) return fail(SCA_EINVAL, "host buffer too small");
    cudaError_t e = cudaMemcpyAsync(host_words, b->state + b->state_off[index], need * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? SCA_OK : cuda_fail(e, "sca_batch_get_state");
}

int sca_batch_set_state(sca_batch *b, uint32_t index, const uint32_t *host_words, size_t n_words)
{
    if (!b || !host_words || index >= b->count) return fail(SCA_EINVAL, "bad argument");
    const uint32_t L = b->lat[index].L;
    const size_t need = (size_t)L * L / 16;
    if (n_words < need) return fail(SCA_EINVAL, "host buffer too small");
    uint32_t *dst = b->state + b->state_off[index];
    uint32_t *scratch = nullptr;
    bool surface = false;
    cudaError_t e = cudaMemcpyAsync(dst, host_words, need * sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&scratch, 4 * sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = surface_check(dst, L, L, scratch, b->stream, &surface);
    if (scratch) {
        const cudaError_t e2 = cudaFreeAsync(scratch, b->stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_batch_set_state");
    if (!surface) {
        // both engines update height bits, exact for surfaces only: back to flat, refused
        const size_t bytes = need * sizeof(uint32_t);
        e = cudaMemsetAsync(dst, 0x00, bytes / 2, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync((char *)dst + bytes / 2, 0xFF, bytes / 2, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        return fail(SCA_ESTATE, "the state is not a surface (a plaquette or row 0 / column 0 does not close)");
    }
    return SCA_OK;
}

uint64_t sca_batch_time(const sca_batch *b) { return b ? b->t : 0; }

int sca_batch_unit_times(sca_batch *b, uint64_t *start_ns, uint64_t *end_ns, int32_t *first_lattice,
                         uint32_t n)
{
    if (!b) return fail(SCA_EINVAL, "NULL batch");
    const uint32_t u = (uint32_t)b->n_units;
    if (n < u) return fail(SCA_EINVAL, "buffers shorter than the unit count");
    std::vector<uint64_t> ns(2 * (size_t)u);
    cudaError_t e = cudaMemcpyAsync(ns.data(), b->unit_ns, ns.size() * sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_batch_unit_times");
    for (uint32_t i = 0; i < u; ++i) {
        if (start_ns) start_ns[i] = ns[2 * i];
        if (end_ns) end_ns[i] = ns[2 * i + 1];
        if (first_lattice) first_lattice[i] = b->unit_first[i];
    }
    return SCA_OK;
}

int sca_batch_tune(sca_batch *b, uint32_t probe_mcs, int *best_cluster, int *best_threads)
{
    if (!b || probe_mcs == 0) return fail(SCA_EINVAL, "bad argument");
    struct Shape { int c, t; size_t cap; };
    // one CTA per SM with up to 200 KiB each, or two per SM with up to 100 KiB (more CTAs
    // per lattice, hence larger clusters)
    const Shape shapes[] = {{8, 512, 200 * 1024}, {6, 512, 200 * 1024}, {6, 384, 200 * 1024},
                            {5, 512, 220 * 1024}, {8, 384, 200 * 1024}, {16, 256, 100 * 1024},
                            {4, 512, 200 * 1024}};
    double best = 1e300;
    Shape bs{b->C, b->threads, b->cap};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(SCA_ECUDA, "cudaEventCreate");
    const int requested = b->engine;
    b->engine = 1;                               // the shapes are the cluster engine's
    batch_drop_graph(b);
    for (const Shape &sh : shapes) {
        if (batch_plan(b, sh.c, sh.t, sh.cap) != SCA_OK) continue;   // shape does not fit: skip
        int rc = sca_batch_reset(b);
        if (rc) break;
        const uint64_t tt = probe_mcs;
        cudaEventRecord(e0, b->stream);
        rc = sca_batch_run(b, &tt, 1, nullptr, nullptr);
        cudaEventRecord(e1, b->stream);
        if (rc) continue;
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            continue;
        if (ms < best) { best = ms; bs = sh; }
    }
    // the streaming engine, when every lattice fits it; automatic choice takes the faster
    int engine = 1;
    if (wb_supported(b)) {
        b->engine = 2;
        batch_drop_graph(b);
        int rc = sca_batch_reset(b);
        const uint64_t tt = probe_mcs;
        cudaEventRecord(e0, b->stream);
        if (!rc) rc = sca_batch_run(b, &tt, 1, nullptr, nullptr);
        cudaEventRecord(e1, b->stream);
        float ms = 0.f;
        if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best) {
            best = ms;
            engine = 2;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->engine = requested == 0 ? engine : requested;
    batch_drop_graph(b);
    int rc = batch_plan(b, bs.c, bs.t, bs.cap);
    if (!rc) rc = sca_batch_reset(b);
    if (rc) return rc;
    if (best_cluster) *best_cluster = bs.c;
    if (best_threads) *best_threads = bs.t;
    return SCA_OK;
}

void sca_batch_free(sca_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    cudaFree(b->state);
    cudaFree(b->lat_d);
    cudaFree(b->slots_d);
    cudaFree(b->counter);
    cudaFree(b->times_d);
    cudaFree(b->unit_ns);
    cudaFree(b->part);
    cudaFree(b->res);
    if (b->res_h) cudaFreeHost(b->res_h);
    wb_free(b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
