// Host runtime of the batched solver (lbms_batch_* in include/lbms.h):
// instance tables, workspace layout, step schedules and their CUDA graphs, the
// schedule tuner, host staging and the per-instance mass reduction.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "batch.cuh"
#include "lbms_internal.h"

using namespace lbms;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStagingMax = size_t(16) << 20;
constexpr int kStreamSteps = 32;  // steps per captured graph of the streamed schedule

// Step schedules the tuner chooses from: 0 streams every instance through HBM
// each step; the others run groups of consecutive instances whose two
// population buffers fit in `budget` bytes for `chunk` steps each, so that a
// group's state stays in the 129 MB L2 between its steps.
struct Candidate {
    size_t budget;
    int chunk;
};
// Candidates of the tuner: schedule c % kSchedules with the kernel shape
// c / kSchedules (0: one node per thread; 1: two nodes per thread, for the
// lattices, species counts and dtypes that have the pair kernel).
constexpr int kSchedules = 7;
static_assert(LBMS_BATCH_CANDIDATES == 2 * kSchedules, "candidates: schedules x kernel shapes");
constexpr Candidate kCandidates[kSchedules] = {
    {0, 0},
    {size_t(24) << 20, 8},  {size_t(24) << 20, 32},
    {size_t(48) << 20, 8},  {size_t(48) << 20, 32},
    {size_t(96) << 20, 8},  {size_t(96) << 20, 32},
};

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int lattice_q(int lat)
{
    switch (lat) {
        case LBMS_D2Q5: return 5;
        case LBMS_D2Q9: return 9;
        case LBMS_D3Q7: return 7;
        case LBMS_D3Q15: return 15;
        case LBMS_D1Q3: return 3;
        case LBMS_D2Q4: return 4;
        case LBMS_D3Q6: return 6;
        default: return 0;
    }
}
int lattice_dim(int lat)
{
    return lat == LBMS_D3Q7 || lat == LBMS_D3Q15 || lat == LBMS_D3Q6 ? 3 : (lat == LBMS_D1Q3 ? 1 : 2);
}

struct BLayout {
    uint32_t total_blocks = 0, total_nodes = 0;
    size_t f_bytes = 0, off_f1 = 0, off_partials = 0, off_mass = 0, off_inst = 0, off_blk = 0,
           off_invD = 0, off_clock = 0, off_foff = 0, off_xb = 0, off_status = 0, off_staging = 0,
           staging_bytes = 0, total = 0;
};

bool batch_layout(int lat, int n, int count, const int* grids, int dtype, BLayout* L)
{
    const int Q = lattice_q(lat);
    if (!Q || n < 2 || n > LBMS_MAX_SPECIES || count < 1 || !grids) return false;
    if (dtype != LBMS_F32 && dtype != LBMS_F64) return false;
    const int dim = lattice_dim(lat);
    double blocks = 0.0, max_field = 0.0;
    for (int i = 0; i < count; ++i) {
        const int* g = grids + 3 * i;
        if (g[0] < 1 || g[1] < 1 || g[2] < 1) return false;
        if (dim < 3 && g[2] != 1) return false;
        if (dim == 1 && g[1] != 1) return false;
        const double c = (double)g[0] * g[1] * g[2];
        if (c > (double)LBMS_MAX_CELLS) return false;
        blocks += ceil(c / kBlock);
        if (c > max_field) max_field = c;
    }
    if (blocks * kBlock > (double)LBMS_MAX_CELLS) return false;
    const size_t es = dtype == LBMS_F64 ? 8 : 4;
    L->total_blocks = (uint32_t)blocks;
    L->total_nodes = L->total_blocks * kBlock;
    L->f_bytes = align_up((size_t)(n - 1) * Q * L->total_nodes * es);
    L->off_f1 = L->f_bytes;
    L->off_partials = 2 * L->f_bytes;
    L->off_mass = L->off_partials + align_up((size_t)L->total_blocks * n * sizeof(double2));
    L->off_inst = L->off_mass + align_up((size_t)count * n * sizeof(double));
    L->off_blk = L->off_inst + align_up((size_t)count * sizeof(BatchInst));
    L->off_invD = L->off_blk + align_up((size_t)L->total_blocks * sizeof(uint32_t));
    L->off_clock = L->off_invD + align_up((size_t)count * n * n * es);
    L->off_foff = L->off_clock + align_up((size_t)count * 2 * sizeof(uint32_t));
    L->off_xb = L->off_foff + align_up((size_t)count * sizeof(long long));
    // Dirichlet compositions [count][6][S]
    L->off_status = L->off_xb + align_up((size_t)count * 6 * (n - 1) * es);
    L->off_staging = L->off_status + kAlign;
    // staging: large enough for the biggest instance's fields, at most 16 MiB beyond that
    const size_t biggest = (size_t)max_field * n * (1 + dim) * es;
    L->staging_bytes = align_up(biggest > kStagingMax ? biggest : kStagingMax);
    L->total = L->off_staging + L->staging_bytes;
    return true;
}

thread_local char g_batch_error[256] = "";

__global__ void k_batch_finalize_fixed(const long long* __restrict__ partials,
                                       const BatchInst* __restrict__ inst, int n, int shift,
                                       double* __restrict__ out)
{
    __shared__ long long red[kBlock / 32];
    const BatchInst d = inst[blockIdx.x];
    for (int s = 0; s < n; ++s) {
        long long acc = 0;
        for (uint32_t b = threadIdx.x; b < d.nblocks; b += blockDim.x)
            acc += partials[(size_t)(d.block0 + b) * n + s];
        const long long tot = block_reduce_fixed(acc, red);
        if (threadIdx.x == 0) out[(size_t)blockIdx.x * n + s] = ldexp((double)tot, -shift);
    }
}

__global__ void k_batch_finalize_pairs(const double2* __restrict__ partials,
                                       const BatchInst* __restrict__ inst, int n,
                                       double* __restrict__ out)
{
    __shared__ double2 red[kBlock / 32];
    const BatchInst d = inst[blockIdx.x];
    for (int s = 0; s < n; ++s) {
        double sum = 0.0, comp = 0.0;
        for (uint32_t b = threadIdx.x; b < d.nblocks; b += blockDim.x) {
            const double2 v = partials[(size_t)(d.block0 + b) * n + s];
            two_sum_merge(sum, comp, v.x, v.y);
        }
        block_reduce_pair(sum, comp, red);
        if (threadIdx.x == 0) out[(size_t)blockIdx.x * n + s] = sum + comp;
    }
}

}  // namespace

struct lbms_batch_s {
    int lattice = 0, n = 0, S = 0, Q = 0, dim = 0, dtype = 0, relax = 0, count = 0;
    size_t es = 4;
    BLayout lay;
    std::vector<BatchInst> inst;
    std::vector<long long> packed_off;  // packed element offsets of the instances' x blocks
    std::vector<long long> off_scratch;
    char* ws = nullptr;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* partials = nullptr;
    double* mass_dev = nullptr;
    bool partials_valid = false;  // the mass partials are those of the current state
    bool mass_valid = false;      // mass_dev holds their reduction
    BatchInst* inst_dev = nullptr;
    uint32_t* blk_dev = nullptr;
    void* invD_dev = nullptr;
    uint32_t* clock = nullptr;
    long long* foff_dev = nullptr;
    void* xb_dev = nullptr;               // [count][6][S] Dirichlet compositions, solver dtype
    std::vector<uint32_t> dirichlet;      // per instance: Dirichlet face mask
    std::vector<uint32_t> xb_set;         // per instance: Dirichlet faces whose composition is set
    bool any_dirichlet = false;
    uint32_t* status = nullptr;
    char* staging = nullptr;
    int fixed_shift = 32;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    int schedule = 0;
    int shape = 0;  // nodes per thread of the plain steps - 1
    std::vector<std::pair<uint32_t, uint32_t>> groups;  // block ranges of the grouped schedule
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long steps = 0;
    char err[512] = "";
};

namespace {

int bfail(lbms_batch_t* b, int code, const char* fmt, ...)
{
    char* buf = b ? b->err : g_batch_error;
    size_t cap = b ? sizeof(b->err) : sizeof(g_batch_error);
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, cap, fmt, ap);
    va_end(ap);
    return code;
}

int bcuda(lbms_batch_t* b, cudaError_t e, const char* what)
{
    return bfail(b, LBMS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t bdispatch(const lbms_batch_t* b, BatchOp op, const BArgs& a)
{
    switch (b->lattice) {
        case LBMS_D2Q5: return batch_dispatch_d2q5(op, b->dtype, a);
        case LBMS_D2Q9: return batch_dispatch_d2q9(op, b->dtype, a);
        case LBMS_D3Q7: return batch_dispatch_d3q7(op, b->dtype, a);
        case LBMS_D3Q15: return batch_dispatch_d3q15(op, b->dtype, a);
        case LBMS_D1Q3: return batch_dispatch_d1q3(op, b->dtype, a);
        case LBMS_D2Q4: return batch_dispatch_d2q4(op, b->dtype, a);
        default: return batch_dispatch_d3q6(op, b->dtype, a);
    }
}

BArgs bargs(const lbms_batch_t* b, cudaStream_t st, uint32_t b0, uint32_t b1)
{
    BArgs a;
    a.total_nodes = b->lay.total_nodes;
    a.block_begin = b0;
    a.block_end = b1;
    a.blk_inst = b->blk_dev;
    a.inst = b->inst_dev;
    a.invD = b->invD_dev;
    a.n_species = b->n;
    a.relax = b->relax;
    a.clock = b->clock;
    a.partials = b->partials;
    a.fixed_shift = b->fixed_shift;
    a.status = b->status;
    a.field_off = b->foff_dev;
    a.xb = b->xb_dev;
    a.dirichlet = b->any_dirichlet;
    a.stream = st;
    return a;
}

cudaError_t bstep(const lbms_batch_t* b, int src, bool mass, uint32_t b0, uint32_t b1,
                  cudaStream_t st)
{
    BArgs a = bargs(b, st, b0, b1);
    a.fin = b->f[src];
    a.fout = b->f[1 - src];
    a.parity = src;
    a.reverse = src;  // alternate steps take the blocks from the end (same-box A/B: +0.35 %)
    a.nodes_per_thread = b->shape + 1;
    return bdispatch(b, mass ? BOP_STEP_MASS : BOP_STEP, a);
}

cudaError_t bfinalize(const lbms_batch_t* b, cudaStream_t st)
{
    if (b->dtype == LBMS_F32)
        k_batch_finalize_fixed<<<b->count, kBlock, 0, st>>>(static_cast<const long long*>(b->partials),
                                                              b->inst_dev, b->n, b->fixed_shift, b->mass_dev);
    else
        k_batch_finalize_pairs<<<b->count, kBlock, 0, st>>>(static_cast<const double2*>(b->partials),
                                                              b->inst_dev, b->n, b->mass_dev);
    return cudaGetLastError();
}

void build_groups(lbms_batch_t* b, size_t budget)
{
    b->groups.clear();
    const size_t per_node = 2 * (size_t)b->S * b->Q * b->es;
    uint32_t g0 = b->inst[0].block0, g1 = g0;
    size_t bytes = 0;
    for (int i = 0; i < b->count; ++i) {
        const size_t ib = (size_t)b->inst[i].nblocks * kBlock * per_node;
        if (g1 > g0 && bytes + ib > budget) {
            b->groups.push_back({g0, g1});
            g0 = g1;
            bytes = 0;
        }
        g1 = b->inst[i].block0 + b->inst[i].nblocks;
        bytes += ib;
    }
    b->groups.push_back({g0, g1});
}

void drop_graphs(lbms_batch_t* b)
{
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

// Whether the batch's steps have a two-nodes-per-thread kernel (ternary or
// binary FP32 solves on the lattices with Q <= 5: D2Q5, D1Q3, D2Q4).
bool has_pair_shape(const lbms_batch_t* b)
{
    return b->Q <= 5 && b->S <= 2 && b->dtype == LBMS_F32;
}

// Steps one graph holds: kStreamSteps for the streamed schedule, one chunk of
// every group for the grouped ones.
int graph_steps(const lbms_batch_t* b)
{
    return b->schedule == 0 ? kStreamSteps : kCandidates[b->schedule].chunk;
}

cudaError_t launch_body(const lbms_batch_t* b, int parity, int steps, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (b->schedule == 0) {
        int src = parity;
        for (int i = 0; i < steps && e == cudaSuccess; ++i, src = 1 - src)
            e = bstep(b, src, false, 0, b->lay.total_blocks, st);
        return e;
    }
    for (const auto& g : b->groups) {
        int src = parity;
        for (int i = 0; i < steps && e == cudaSuccess; ++i, src = 1 - src)
            e = bstep(b, src, false, g.first, g.second, st);
    }
    return e;
}

cudaError_t build_graph(lbms_batch_t* b, int parity)
{
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = launch_body(b, parity, graph_steps(b), b->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    return e;
}

bool is_dev(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const long long* user_offsets(lbms_batch_t* b, const int64_t* offsets)
{
    return offsets ? reinterpret_cast<const long long*>(offsets) : b->packed_off.data();
}

}  // namespace

extern "C" {

size_t lbms_batch_workspace_size(int lattice, int n_species, int count, const int* grids, int dtype)
{
    BLayout L;
    return batch_layout(lattice, n_species, count, grids, dtype, &L) ? L.total : 0;
}

int lbms_batch_create(lbms_batch_t** out, int lattice, int n_species, int count, const int* grids,
                      const double* D, int relax, const int* bc, int dtype, void* workspace,
                      size_t workspace_bytes, void* cuda_stream)
{
    g_batch_error[0] = '\0';
    if (!out) return bfail(nullptr, LBMS_EINVAL, "out is NULL");
    *out = nullptr;
    BLayout L;
    if (!batch_layout(lattice, n_species, count, grids, dtype, &L))
        return bfail(nullptr, LBMS_EINVAL, "invalid lattice/species/count/grids/dtype combination");
    if (relax != LBMS_RELAX_MAGIC && relax != LBMS_RELAX_SRT)
        return bfail(nullptr, LBMS_EINVAL, "invalid relaxation mode %d", relax);
    if (!D) return bfail(nullptr, LBMS_EINVAL, "D is NULL");
    if (!workspace || (uintptr_t)workspace % kAlign)
        return bfail(nullptr, LBMS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (workspace_bytes < L.total)
        return bfail(nullptr, LBMS_ENOMEM, "workspace holds %zu bytes, %zu needed", workspace_bytes, L.total);
    const int n = n_species, dim = lattice_dim(lattice);
    for (int c = 0; c < count; ++c) {
        const double* Dc = D + (size_t)c * n * n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j) continue;
                const double d = Dc[i * n + j];
                if (!(isfinite(d) && d > 0.0))
                    return bfail(nullptr, LBMS_EINVAL, "instance %d: D[%d][%d] = %g is not finite and positive",
                                 c, i, j, d);
                if (d != Dc[j * n + i])
                    return bfail(nullptr, LBMS_EINVAL, "instance %d: D is not symmetric", c);
            }
        if (bc)
            for (int a = 0; a < dim; ++a) {
                const int lo = bc[6 * c + 2 * a], hi = bc[6 * c + 2 * a + 1];
                if (lo < LBMS_PERIODIC || lo > LBMS_DIRICHLET || hi < LBMS_PERIODIC || hi > LBMS_DIRICHLET ||
                    ((lo == LBMS_PERIODIC) != (hi == LBMS_PERIODIC)))
                    return bfail(nullptr, LBMS_EINVAL, "instance %d: invalid or unpaired faces on axis %d", c, a);
            }
    }
    lbms_batch_t* b = new (std::nothrow) lbms_batch_t;
    if (!b) return bfail(nullptr, LBMS_ENOMEM, "host allocation failed");
    b->lattice = lattice;
    b->n = n;
    b->S = n - 1;
    b->Q = lattice_q(lattice);
    b->dim = dim;
    b->dtype = dtype;
    b->relax = relax;
    b->count = count;
    b->es = dtype == LBMS_F64 ? 8 : 4;
    b->shape = has_pair_shape(b) ? 1 : 0;  // the faster shape where it exists
    b->lay = L;
    b->ws = static_cast<char*>(workspace);
    b->f[0] = b->ws;
    b->f[1] = b->ws + L.off_f1;
    b->partials = b->ws + L.off_partials;
    b->mass_dev = reinterpret_cast<double*>(b->ws + L.off_mass);
    b->inst_dev = reinterpret_cast<BatchInst*>(b->ws + L.off_inst);
    b->blk_dev = reinterpret_cast<uint32_t*>(b->ws + L.off_blk);
    b->invD_dev = b->ws + L.off_invD;
    b->clock = reinterpret_cast<uint32_t*>(b->ws + L.off_clock);
    b->foff_dev = reinterpret_cast<long long*>(b->ws + L.off_foff);
    b->xb_dev = b->ws + L.off_xb;
    b->dirichlet.assign(count, 0u);
    b->xb_set.assign(count, 0u);
    b->status = reinterpret_cast<uint32_t*>(b->ws + L.off_status);
    b->staging = b->ws + L.off_staging;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    uint32_t maxcells = 0;
    // host tables
    b->inst.resize(count);
    b->packed_off.resize(count);
    std::vector<uint32_t> blk(L.total_blocks);
    std::vector<char> invD((size_t)count * n * n * b->es);
    uint32_t block = 0;
    long long off = 0;
    for (int c = 0; c < count; ++c) {
        KArgs ka;
        ka.nx = grids[3 * c]; ka.ny = grids[3 * c + 1]; ka.nz = grids[3 * c + 2];
        ka.cells = (uint32_t)((size_t)ka.nx * ka.ny * ka.nz);
        uint32_t nf = 0, dr = 0;
        if (bc)
            for (int a = 0; a < dim; ++a) {
                if (bc[6 * c + 2 * a] == LBMS_NOFLUX) nf |= 1u << (2 * a);
                if (bc[6 * c + 2 * a + 1] == LBMS_NOFLUX) nf |= 1u << (2 * a + 1);
                if (bc[6 * c + 2 * a] == LBMS_DIRICHLET) dr |= 1u << (2 * a);
                if (bc[6 * c + 2 * a + 1] == LBMS_DIRICHLET) dr |= 1u << (2 * a + 1);
            }
        ka.noflux = nf;
        ka.dirichlet = dr;
        b->dirichlet[c] = dr;
        b->any_dirichlet |= dr != 0;
        BatchInst& d = b->inst[c];
        d.g = make_geom(ka);
        d.base = block * kBlock;
        d.block0 = block;
        d.nblocks = node_blocks(ka.cells);
        d.pad = 0;
        for (uint32_t k = 0; k < d.nblocks; ++k) blk[block + k] = (uint32_t)c;
        block += d.nblocks;
        b->packed_off[c] = off;
        off += (long long)n * ka.cells;
        if (ka.cells > maxcells) maxcells = ka.cells;
        const double* Dc = D + (size_t)c * n * n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                // halved inverse diffusivities (relaxation_matrices takes 1/(2 D_ij))
                const double v = i == j ? 0.0 : 0.5 * (1.0 / Dc[i * n + j]);
                const size_t at = ((size_t)c * n * n + i * n + j);
                if (dtype == LBMS_F64)
                    reinterpret_cast<double*>(invD.data())[at] = v;
                else
                    reinterpret_cast<float*>(invD.data())[at] = (float)v;
            }
    }
    // the fixed-point resolution follows the largest instance (per-instance sums)
    int l = 0;
    while ((1ull << l) < maxcells) ++l;
    int k = 62 - l - 3;
    b->fixed_shift = k > 40 ? 40 : (k < 8 ? 8 : k);
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->inst_dev, b->inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->blk_dev, blk.data(), sizeof(uint32_t) * blk.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->invD_dev, invD.data(), invD.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->clock, 0, sizeof(uint32_t) * 2 * count, b->stream);
    // the host tables are copied from pageable memory: wait before they go
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        if (b->capture) cudaStreamDestroy(b->capture);
        delete b;
        return bfail(nullptr, LBMS_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    }
    *out = b;
    return LBMS_OK;
}

int lbms_batch_set_state(lbms_batch_t* b, const void* x0, const int64_t* offsets)
{
    if (!b) return LBMS_EINVAL;
    if (!x0) return bfail(b, LBMS_EINVAL, "x0 is NULL");
    b->err[0] = '\0';
    cudaError_t e = cudaMemsetAsync(b->status, 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->clock, 0, sizeof(uint32_t) * 2 * b->count, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync");
    b->cur = 0;
    b->steps = 0;
    b->partials_valid = false;
    b->mass_valid = false;
    const long long* uoff = user_offsets(b, offsets);
    BArgs a = bargs(b, b->stream, 0, b->lay.total_blocks);
    a.fout = b->f[0];
    const void* alias = pinned_alias(x0);
    if (alias || is_dev(x0)) {
        // device memory, or pinned host memory read by the kernel in place
        e = cudaMemcpyAsync(b->foff_dev, uoff, sizeof(long long) * b->count, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "offset upload");
        a.field_in = alias ? alias : x0;
        e = bdispatch(b, BOP_INIT, a);
        if (e == cudaSuccess && alias) e = cudaStreamSynchronize(b->stream);  // x0 is free on return
        return e == cudaSuccess ? LBMS_OK : bcuda(b, e, "batch init kernel");
    }
    // host source: pack consecutive instances into the staging area
    b->off_scratch.assign(b->count, 0);
    const char* src = static_cast<const char*>(x0);
    int i0 = 0;
    while (i0 < b->count) {
        size_t used = 0;
        int i1 = i0;
        while (i1 < b->count) {
            const size_t bytes = (size_t)b->n * b->inst[i1].g.cells * b->es;
            if (i1 > i0 && used + bytes > b->lay.staging_bytes) break;
            e = cudaMemcpyAsync(b->staging + used, src + uoff[i1] * b->es, bytes, cudaMemcpyHostToDevice,
                                b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync (host to device)");
            b->off_scratch[i1] = (long long)(used / b->es);
            used += bytes;
            ++i1;
        }
        e = cudaMemcpyAsync(b->foff_dev + i0, b->off_scratch.data() + i0, sizeof(long long) * (i1 - i0),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "offset upload");
        a.field_in = b->staging;
        a.block_begin = b->inst[i0].block0;
        a.block_end = b->inst[i1 - 1].block0 + b->inst[i1 - 1].nblocks;
        e = bdispatch(b, BOP_INIT, a);
        if (e != cudaSuccess) return bcuda(b, e, "batch init kernel");
        // the next pack reuses the staging area and the offset words: wait
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
        i0 = i1;
    }
    return LBMS_OK;
}

int lbms_batch_step(lbms_batch_t* b, long n_steps)
{
    if (!b) return LBMS_EINVAL;
    if (n_steps < 0) return bfail(b, LBMS_EINVAL, "n_steps = %ld is negative", n_steps);
    for (int c = 0; c < b->count; ++c)
        if (b->dirichlet[c] & ~b->xb_set[c])
            return bfail(b, LBMS_EINVAL, "instance %d: Dirichlet face mask 0x%x has no composition set", c,
                         b->dirichlet[c] & ~b->xb_set[c]);
    b->err[0] = '\0';
    if (n_steps == 0) return LBMS_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(b->stream, &cs);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamIsCapturing");
    const int gs = graph_steps(b);
    long body = n_steps - 1;
    if (cs == cudaStreamCaptureStatusNone) {
        while (body >= gs) {
            if (!b->graph[b->cur]) {
                e = build_graph(b, b->cur);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    break;  // direct launches below
                }
            }
            e = cudaGraphLaunch(b->graph[b->cur], b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
            if (gs & 1) b->cur = 1 - b->cur;
            body -= gs;
            b->steps += gs;
        }
    }
    while (body > 0) {
        const int chunk = (int)(body < gs ? body : gs);
        e = launch_body(b, b->cur, chunk, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "batch step kernel");
        if (chunk & 1) b->cur = 1 - b->cur;
        body -= chunk;
        b->steps += chunk;
    }
    e = bstep(b, b->cur, true, 0, b->lay.total_blocks, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch step kernel");
    b->cur = 1 - b->cur;
    ++b->steps;
    // the reduction of the partials waits for lbms_batch_mass
    b->partials_valid = true;
    b->mass_valid = false;
    return LBMS_OK;
}

int lbms_batch_moments(lbms_batch_t* b, void* x_sigma, void* J_sigma, const int64_t* offsets)
{
    if (!b) return LBMS_EINVAL;
    if (!x_sigma) return bfail(b, LBMS_EINVAL, "x_sigma is NULL");
    b->err[0] = '\0';
    const long long* uoff = user_offsets(b, offsets);
    BArgs a = bargs(b, b->stream, 0, b->lay.total_blocks);
    a.fin = b->steps > 0 ? b->f[1 - b->cur] : nullptr;
    a.fout = b->f[b->cur];
    // device memory, or pinned host memory written by the kernel in place
    void* xalias = pinned_alias(x_sigma);
    void* jalias = J_sigma ? pinned_alias(J_sigma) : nullptr;
    const bool xdev = xalias || is_dev(x_sigma), jdev = J_sigma ? (jalias || is_dev(J_sigma)) : true;
    cudaError_t e;
    if (xdev && jdev) {
        e = cudaMemcpyAsync(b->foff_dev, uoff, sizeof(long long) * b->count, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "offset upload");
        a.field_x = xalias ? xalias : x_sigma;
        a.field_J = jalias ? jalias : J_sigma;
        e = bdispatch(b, BOP_MOMENTS, a);
        if (e != cudaSuccess) return bcuda(b, e, "batch moments kernel");
        e = cudaStreamSynchronize(b->stream);  // the offsets came from pageable memory
        return e == cudaSuccess ? LBMS_OK : bcuda(b, e, "cudaStreamSynchronize");
    }
    const size_t mult = 1 + (J_sigma ? b->dim : 0);
    b->off_scratch.assign(b->count, 0);
    char* xo = static_cast<char*>(x_sigma);
    char* jo = static_cast<char*>(J_sigma);
    int i0 = 0;
    while (i0 < b->count) {
        size_t used = 0;  // elements of x in this pack; J follows at dim * used
        int i1 = i0;
        while (i1 < b->count) {
            const size_t el = (size_t)b->n * b->inst[i1].g.cells;
            if (i1 > i0 && (used + el) * mult * b->es > b->lay.staging_bytes) break;
            b->off_scratch[i1] = (long long)used;
            used += el;
            ++i1;
        }
        e = cudaMemcpyAsync(b->foff_dev + i0, b->off_scratch.data() + i0, sizeof(long long) * (i1 - i0),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "offset upload");
        a.field_x = b->staging;
        a.field_J = J_sigma ? b->staging + used * b->es : nullptr;
        a.block_begin = b->inst[i0].block0;
        a.block_end = b->inst[i1 - 1].block0 + b->inst[i1 - 1].nblocks;
        e = bdispatch(b, BOP_MOMENTS, a);
        if (e != cudaSuccess) return bcuda(b, e, "batch moments kernel");
        for (int i = i0; i < i1; ++i) {
            const size_t el = (size_t)b->n * b->inst[i].g.cells;
            e = cudaMemcpyAsync(xo + uoff[i] * b->es, b->staging + b->off_scratch[i] * b->es, el * b->es,
                                cudaMemcpyDefault, b->stream);
            if (e == cudaSuccess && J_sigma)
                e = cudaMemcpyAsync(jo + (size_t)b->dim * uoff[i] * b->es,
                                    b->staging + (used + (size_t)b->dim * b->off_scratch[i]) * b->es,
                                    el * b->dim * b->es, cudaMemcpyDefault, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync (moments)");
        }
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
        i0 = i1;
    }
    return LBMS_OK;
}

int lbms_batch_mass(lbms_batch_t* b, double* mass_out)
{
    if (!b) return LBMS_EINVAL;
    if (!mass_out) return bfail(b, LBMS_EINVAL, "mass_out is NULL");
    b->err[0] = '\0';
    cudaError_t e;
    if (!b->partials_valid) {
        BArgs a = bargs(b, b->stream, 0, b->lay.total_blocks);
        a.fout = b->f[b->cur];
        e = bdispatch(b, BOP_MASS, a);
        if (e != cudaSuccess) return bcuda(b, e, "batch mass kernel");
        b->partials_valid = true;
        b->mass_valid = false;
    }
    if (!b->mass_valid) {
        e = bfinalize(b, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "batch mass reduction");
        b->mass_valid = true;
    }
    e = cudaMemcpyAsync(mass_out, b->mass_dev, sizeof(double) * b->count * b->n, cudaMemcpyDeviceToHost,
                        b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? LBMS_OK : bcuda(b, e, "mass copy");
}

int lbms_batch_status(lbms_batch_t* b, uint32_t* flags)
{
    if (!b || !flags) return LBMS_EINVAL;
    cudaError_t e = cudaMemcpyAsync(flags, b->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? LBMS_OK : bcuda(b, e, "status copy");
}

int lbms_batch_set_boundary(lbms_batch_t* b, int instance, int face, const double* xi_b)
{
    if (!b) return LBMS_EINVAL;
    if (instance < 0 || instance >= b->count) return bfail(b, LBMS_EINVAL, "instance %d out of range", instance);
    if (face < 0 || face > 5 || !((b->dirichlet[instance] >> face) & 1u))
        return bfail(b, LBMS_EINVAL, "instance %d: face %d is not a Dirichlet face", instance, face);
    if (!xi_b) return bfail(b, LBMS_EINVAL, "xi_b is NULL");
    double sum = 0.0;
    for (int s = 0; s < b->n; ++s) {
        if (!isfinite(xi_b[s]) || xi_b[s] < -1e-6 || xi_b[s] > 1.0 + 1e-6)
            return bfail(b, LBMS_EINVAL, "xi_b[%d] = %g is not a mole fraction", s, xi_b[s]);
        sum += xi_b[s];
    }
    if (fabs(sum - 1.0) > 1e-6) return bfail(b, LBMS_EINVAL, "the composition sums to %.9g, not 1", sum);
    b->err[0] = '\0';
    double v64[LBMS_MAX_SPECIES];
    float v32[LBMS_MAX_SPECIES];
    for (int s = 0; s < b->S; ++s) {
        v64[s] = xi_b[s];
        v32[s] = (float)xi_b[s];
    }
    const void* src = b->dtype == LBMS_F64 ? static_cast<const void*>(v64) : static_cast<const void*>(v32);
    char* dst = static_cast<char*>(b->xb_dev) + ((size_t)instance * 6 + face) * b->S * b->es;
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)b->S * b->es, cudaMemcpyHostToDevice, b->stream);
    // the copy reads pageable memory: wait for it before the locals go away
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "boundary composition copy");
    b->xb_set[instance] |= 1u << face;
    return LBMS_OK;
}

int lbms_batch_set_schedule(lbms_batch_t* b, int candidate)
{
    if (!b) return LBMS_EINVAL;
    if (candidate < 0 || candidate >= LBMS_BATCH_CANDIDATES)
        return bfail(b, LBMS_EINVAL, "schedule %d is not one of 0..%d", candidate, LBMS_BATCH_CANDIDATES - 1);
    const int schedule = candidate % kSchedules, shape = candidate / kSchedules;
    if (shape == 1 && !has_pair_shape(b))
        return bfail(b, LBMS_EINVAL, "candidate %d needs the two-nodes-per-thread kernel (Q <= 5, n <= 3, F32)",
                     candidate);
    if (schedule == b->schedule && shape == b->shape) return LBMS_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
    drop_graphs(b);
    b->schedule = schedule;
    b->shape = shape;
    if (schedule > 0) build_groups(b, kCandidates[schedule].budget);
    return LBMS_OK;
}

int lbms_batch_get_schedule(const lbms_batch_t* b) { return b ? b->schedule + kSchedules * b->shape : -1; }

int lbms_batch_launches_per_step(const lbms_batch_t* b)
{
    if (!b) return -1;
    return b->schedule == 0 ? 1 : (int)b->groups.size();
}

int lbms_batch_tune(lbms_batch_t* b, int trial_steps, double* ms_per_step, int* chosen)
{
    if (!b) return LBMS_EINVAL;
    if (trial_steps < 2) return bfail(b, LBMS_EINVAL, "trial_steps must be at least 2");
    double best = 1e300;
    int best_c = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return bcuda(b, e, "cudaEventCreate");
    int rc = LBMS_OK;
    for (int c = 0; c < LBMS_BATCH_CANDIDATES && rc == LBMS_OK; ++c) {
        if (c / kSchedules == 1 && !has_pair_shape(b)) {
            if (ms_per_step) ms_per_step[c] = -1.0;  // not available for this batch
            continue;
        }
        rc = lbms_batch_set_schedule(b, c);
        if (rc == LBMS_OK) rc = lbms_batch_step(b, trial_steps);  // warm-up, builds the graphs
        if (rc != LBMS_OK) break;
        e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess && lbms_batch_step(b, trial_steps) != LBMS_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = bcuda(b, e, "tuner timing");
            break;
        }
        const double per = ms / trial_steps;
        if (ms_per_step) ms_per_step[c] = per;
        if (per < best) {
            best = per;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBMS_OK) return rc;
    rc = lbms_batch_set_schedule(b, best_c);
    if (chosen) *chosen = best_c;
    return rc;
}

long lbms_batch_steps_done(const lbms_batch_t* b) { return b ? b->steps : -1; }

const char* lbms_batch_last_error(const lbms_batch_t* b) { return b ? b->err : g_batch_error; }

void lbms_batch_destroy(lbms_batch_t* b)
{
    if (!b) return;
    drop_graphs(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

}  // extern "C"
