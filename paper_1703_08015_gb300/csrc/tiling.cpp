// tiling.cpp -- host-side tiling of a masked lattice (Sec. 3 of
// Tomczak & Szafran, arXiv:1703.08015) and the lbm_build_tilemap entry point.
//
// The geometry is covered by a uniform mesh of a x a (x a) tiles anchored at
// node (0,0); nodes beyond the lattice are solid padding; tiles with no fluid
// node are removed.  A non-empty tile's index is its rank in row-major scan
// order (x fastest), which is what the tileMap stores (-1 for removed tiles).
// Each non-empty tile also gets the 3^d record of its neighbours' indices
// (the local copy of the tile bitmap in Fig. 5) and a bit mask of its fluid
// nodes (one bit per node instead of the paper's s_t = 2 bytes, Eq. 21).
// PDFs are stored compactly: a tile's block holds only its fluid nodes (in
// row order), so solid nodes of porous tiles cost neither memory nor
// bandwidth; a node's slot is its rank among the tile's fluid nodes.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>

#include "internal.h"

namespace lbm {

// Host threads for the tiling, started once per process (the calling
// thread takes a share too): starting threads for every parallel pass cost
// about 0.4 ms per pass on the Grace host, more than most passes' work.  The
// workers sleep on a condition variable between calls; one call uses the pool
// at a time (a concurrent call runs serially), and a forked child, which has
// no copy of the workers, starts its own pool.
struct HostPool {
    std::mutex mu, busy;
    std::condition_variable work_cv, done_cv;
    const std::function<void(int64_t, int64_t)>* job = nullptr;
    int64_t n = 0, chunk = 0;
    int n_chunks = 0, next = 0, remaining = 0;
    int threads = 1;  // workers + the caller
    pid_t pid = 0;

    // take chunks until none is left; returns with `lk` held
    void run_chunks(std::unique_lock<std::mutex>& lk) {
        while (next < n_chunks) {
            const int c = next++;
            const int64_t b = (int64_t)c * chunk, e = std::min(n, b + chunk);
            lk.unlock();
            (*job)(b, e);
            lk.lock();
            if (--remaining == 0) done_cv.notify_all();
        }
    }
    void worker() {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            work_cv.wait(lk, [&] { return next < n_chunks; });
            run_chunks(lk);
        }
    }
};

static HostPool* host_pool() {
    static std::mutex init;
    static HostPool* pool = nullptr;
    std::lock_guard<std::mutex> g(init);
    if (pool && pool->pid == getpid()) return pool;
    // first use, or a forked child: a new pool (a parent's is left as it is)
    HostPool* p = new HostPool();
    p->pid = getpid();
    const unsigned hc = std::thread::hardware_concurrency();
    const int want = (int)std::max(1u, std::min(hc ? hc : 1u, 16u));
    for (int k = 1; k < want; k++) {
        try {
            std::thread(&HostPool::worker, p).detach();
            p->threads++;
        } catch (...) {
            break;
        }
    }
    pool = p;
    return pool;
}

// f(begin, end) over [0, n) in up to 16 host threads (each range a contiguous
// block of items; the caller's results depend only on the item, not on the
// split).  Runs serially for small n or while another call holds the pool.
template <class F>
static void parallel_ranges(int64_t n, int64_t min_per_thread, F f) {
    HostPool* P = host_pool();
    const int64_t t = std::min<int64_t>(P->threads, n / std::max<int64_t>(min_per_thread, 1));
    std::unique_lock<std::mutex> busy(P->busy, std::try_to_lock);
    if (t <= 1 || !busy.owns_lock()) {
        f((int64_t)0, n);
        return;
    }
    const std::function<void(int64_t, int64_t)> job = f;
    std::unique_lock<std::mutex> lk(P->mu);
    P->job = &job;
    P->n = n;
    P->chunk = (n + t - 1) / t;
    P->n_chunks = (int)((n + P->chunk - 1) / P->chunk);
    P->next = 0;
    P->remaining = P->n_chunks;
    P->work_cv.notify_all();
    P->run_chunks(lk);
    P->done_cv.wait(lk, [&] { return P->remaining == 0; });
    P->job = nullptr;
}

static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s (%s)", what,
         cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

int lattice_q(int lattice) { return lattice == LBM_D2Q9 ? 9 : lattice == LBM_D3Q19 ? 19 : 0; }

size_t bytes_per_value(int storage) {
    switch (storage) {
        case LBM_STORE_F64: return 8;
        case LBM_STORE_F32: return 4;
        case LBM_STORE_F32S: return 4;
        case LBM_STORE_F16S: return 2;
        default: return 0;
    }
}

static bool tile_edge_ok(int lattice, int a) {
    if (lattice == LBM_D2Q9) return a == 8 || a == 16 || a == 32;
    if (lattice == LBM_D3Q19) return a == 4 || a == 8;
    return false;
}

int validate_params(const lbm_params* p) {
    if (!p) return fail(LBM_ERR_ARG, "params is NULL");
    if (!lattice_q(p->lattice)) return fail(LBM_ERR_ARG, "unknown lattice %d", p->lattice);
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_ERR_ARG, "lattice size must be positive");
    if (p->lattice == LBM_D2Q9 && p->nz != 1) return fail(LBM_ERR_ARG, "D2Q9 needs nz == 1");
    if (!tile_edge_ok(p->lattice, p->tile_a))
        return fail(LBM_ERR_ARG, "tile edge %d not supported for lattice %d", p->tile_a, p->lattice);
    if (!bytes_per_value(p->storage)) return fail(LBM_ERR_ARG, "unknown storage %d", p->storage);
    if (p->model != LBM_QUASI_COMPRESSIBLE && p->model != LBM_INCOMPRESSIBLE)
        return fail(LBM_ERR_ARG, "unknown model %d", p->model);
    if (p->arith < LBM_ARITH_AUTO || p->arith > LBM_ARITH_FF_TABLE)
        return fail(LBM_ERR_ARG, "unknown arithmetic %d", p->arith);
    const int d = p->lattice == LBM_D2Q9 ? 2 : 3;
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int ax = 0; ax < d; ax++)
        if (p->periodic[ax] && n[ax] % p->tile_a != 0)
            return fail(LBM_ERR_SHAPE, "periodic axis %d of length %d is not a multiple of %d", ax,
                        n[ax], p->tile_a);
    return LBM_OK;
}

int build_tiling(const lbm_params* p, const uint8_t* mask, HostTiling* T, bool host_nbr) {
    int rc = validate_params(p);
    if (rc) return rc;
    if (!mask) return fail(LBM_ERR_ARG, "mask is NULL");
    const int a = p->tile_a;
    const int d = p->lattice == LBM_D2Q9 ? 2 : 3;
    const int az = d == 3 ? a : 1;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int ntx = (nx + a - 1) / a, nty = (ny + a - 1) / a, ntz = d == 3 ? (nz + a - 1) / a : 1;
    const int64_t n_tiles64 = (int64_t)ntx * nty * ntz;
    if (n_tiles64 > INT32_MAX) return fail(LBM_ERR_CAPACITY, "too many tiles");
    if (n_tiles64 * a * a * (d == 3 ? a : 1) > (int64_t)UINT32_MAX)
        return fail(LBM_ERR_CAPACITY, "too many tile slots for 32-bit node indices");
    const int nt = a * a * az;
    T->a = a;
    T->d = d;
    T->nn = d == 3 ? 27 : 9;
    T->words = (nt + 63) / 64;
    T->tile_map.assign((size_t)n_tiles64, -1);
    T->nbr.clear();
    T->tmask.clear();
    T->coords.clear();

    // fluid bits and counts of every tile, tile rows (tz, ty) in parallel: each
    // mask row is read once, left to right, its nodes' bits set in the tiles
    // they fall in (node lx + a (ly + a lz) of the tile)
    const int W = T->words;
    int la = 0;
    while ((1 << la) < a) la++;  // a is a power of two (checked by validate_params)
    fill_vector<uint64_t> all_bits((size_t)n_tiles64 * W);  // zeroed row by row below
    fill_vector<int32_t> all_nf((size_t)n_tiles64);
    parallel_ranges((int64_t)ntz * nty, 8, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; r++) {
            const int tz = (int)(r / nty), ty = (int)(r % nty);
            uint64_t* bits = &all_bits[(size_t)r * ntx * W];
            std::memset(bits, 0, (size_t)ntx * W * sizeof(uint64_t));
            for (int lz = 0; lz < az; lz++) {
                const int z = tz * az + lz;
                if (z >= nz) break;
                for (int ly = 0; ly < a; ly++) {
                    const int y = ty * a + ly;
                    if (y >= ny) break;
                    const uint8_t* row = mask + ((size_t)z * ny + y) * nx;
                    const int base = a * (ly + a * lz);  // node index of lx = 0
                    int x = 0;
                    // eight mask bytes at a time: one bit per nonzero byte
                    // (x = 8k: the eight nodes lie in one tile for a >= 8, in
                    // two consecutive tiles for a = 4)
                    for (; x + 8 <= nx; x += 8) {
                        uint64_t v;
                        std::memcpy(&v, row + x, 8);
                        if (!v) continue;
                        const uint64_t hi = ((v & 0x7F7F7F7F7F7F7F7Full) + 0x7F7F7F7F7F7F7F7Full) | v;
                        const uint64_t b8 = (((hi & 0x8080808080808080ull) >> 7) * 0x0102040810204080ull) >> 56;
                        for (int h = 0; h < 8; h += a < 8 ? a : 8) {
                            const uint64_t part = (b8 >> h) & (a < 8 ? (1ull << a) - 1 : 0xFFull);
                            if (!part) continue;
                            const int node = base + ((x + h) & (a - 1));
                            bits[(size_t)((x + h) >> la) * W + (node >> 6)] |= part << (node & 63);
                        }
                    }
                    for (; x < nx; x++) {
                        if (!row[x]) continue;
                        const int node = base + (x & (a - 1));
                        bits[(size_t)(x >> la) * W + (node >> 6)] |= 1ull << (node & 63);
                    }
                }
            }
            for (int tx = 0; tx < ntx; tx++) {
                int nf = 0;
                for (int w = 0; w < W; w++) nf += __builtin_popcountll(bits[(size_t)tx * W + w]);
                all_nf[(size_t)r * ntx + tx] = nf;
            }
        }
    });
    // ranks in row-major scan order: the tile index is a prefix count over the
    // tiles, taken per tile row in parallel, then the rows' offsets
    const int64_t n_rows = (int64_t)ntz * nty;
    std::vector<int32_t> row_count((size_t)n_rows + 1, 0);
    std::vector<int64_t> row_fluid((size_t)n_rows + 1, 0);
    parallel_ranges(n_rows, 64, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; r++) {
            int c = 0;
            int64_t f = 0;
            for (int tx = 0; tx < ntx; tx++) {
                const int32_t nf = all_nf[(size_t)r * ntx + tx];
                c += nf > 0;
                f += nf;
            }
            row_count[r + 1] = c;
            row_fluid[r + 1] = f;
        }
    });
    for (int64_t r = 0; r < n_rows; r++) {
        row_count[r + 1] += row_count[r];
        row_fluid[r + 1] += row_fluid[r];
    }
    const int32_t count = row_count[n_rows];
    const int64_t n_fluid = row_fluid[n_rows];
    T->tmask.resize((size_t)count * W);
    T->coords.resize((size_t)count * 3);
    parallel_ranges(n_rows, 64, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; r++) {
            int32_t k = row_count[r];
            for (int tx = 0; tx < ntx; tx++) {
                const size_t t = (size_t)r * ntx + tx;
                if (!all_nf[t]) continue;
                T->tile_map[t] = k;
                std::memcpy(&T->tmask[(size_t)k * W], &all_bits[t * W], (size_t)W * sizeof(uint64_t));
                T->coords[(size_t)3 * k] = tx;
                T->coords[(size_t)3 * k + 1] = (int)(r % nty);
                T->coords[(size_t)3 * k + 2] = (int)(r / nty);
                k++;
            }
        }
    });

    // neighbour records through a tile map padded by one tile on each side:
    // the pad holds the wrapped tile on a periodic axis, -1 beyond a wall
    // (without host_nbr the caller builds them on the device from tile_map)
    const int per[3] = {p->periodic[0] ? 1 : 0, p->periodic[1] ? 1 : 0, d == 3 && p->periodic[2] ? 1 : 0};
    if (host_nbr) {
        const int ntv[3] = {ntx, nty, ntz};
        const int px = ntx + 2, py = nty + 2, pz = d == 3 ? ntz + 2 : 1;
        std::vector<int32_t> pmap((size_t)px * py * pz, -1);
        parallel_ranges(pz, 4, [&](int64_t z0, int64_t z1) {
            for (int64_t zz = z0; zz < z1; zz++)
                for (int yy = 0; yy < py; yy++)
                    for (int xx = 0; xx < px; xx++) {
                        int q[3] = {xx - 1, yy - 1, d == 3 ? (int)zz - 1 : 0};
                        bool ok = true;
                        for (int ax = 0; ax < d; ax++) {
                            if (q[ax] < 0 || q[ax] >= ntv[ax]) {
                                if (per[ax])
                                    q[ax] = (q[ax] + ntv[ax]) % ntv[ax];
                                else
                                    ok = false;
                            }
                        }
                        pmap[((size_t)zz * py + yy) * px + xx] =
                            ok ? T->tile_map[((size_t)q[2] * nty + q[1]) * ntx + q[0]] : -1;
                    }
        });
        int64_t off[27];
        {
            int slot = 0;
            for (int dz = (d == 3 ? -1 : 0); dz <= (d == 3 ? 1 : 0); dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++, slot++) off[slot] = ((int64_t)dz * py + dy) * px + dx;
        }
        T->nbr.resize((size_t)count * T->nn);
        parallel_ranges(count, 1024, [&](int64_t k0, int64_t k1) {
            for (int64_t k = k0; k < k1; k++) {
                const int* c = &T->coords[(size_t)3 * k];
                const int64_t centre = ((int64_t)(d == 3 ? c[2] + 1 : 0) * py + (c[1] + 1)) * px + (c[0] + 1);
                int32_t* out = &T->nbr[(size_t)k * T->nn];
                for (int slot = 0; slot < T->nn; slot++) out[slot] = pmap[(size_t)(centre + off[slot])];
            }
        });
    }

    // Compact layout: a tile stores only its fluid nodes, in row order, link
    // after link with no padding (contiguous link arrays fill whole sectors).
    const int bpv = (int)bytes_per_value(p->storage);
    constexpr int pad = 1;
    // (pad = 1: a tile's stride is its fluid count, so the offsets are q times
    // the prefix counts of fluid nodes, taken per tile row from the row sums)
    T->tile_off.resize(count);
    T->tile_stride.resize(count);
    const int q = lattice_q(p->lattice);
    static_assert(pad == 1, "offsets from the fluid prefix counts assume no padding");
    parallel_ranges(n_rows, 64, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; r++) {
            int32_t k = row_count[r];
            long long off = (long long)q * row_fluid[r];
            for (int tx = 0; tx < ntx; tx++) {
                const int32_t nf = all_nf[(size_t)r * ntx + tx];
                if (!nf) continue;
                T->tile_off[k] = off;
                T->tile_stride[k] = nf;
                off += (long long)q * nf;
                k++;
            }
        }
    });
    const long long total = (long long)q * n_fluid;

    // the step kernels address a tile's neighbours with 32-bit value offsets
    // from the first tile of their block: neighbours must lie within 2^30
    // values (always so when the whole copy holds fewer values)
    std::atomic<bool> far{false};
    if (host_nbr && total > (1ll << 30)) parallel_ranges(count, 4096, [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1 && !far.load(std::memory_order_relaxed); k++)
            for (int slot = 0; slot < T->nn; slot++) {
                const int32_t nb = T->nbr[(size_t)k * T->nn + slot];
                if (nb >= 0 && std::llabs(T->tile_off[nb] - T->tile_off[k]) > (1ll << 30))
                    far.store(true, std::memory_order_relaxed);
            }
    });
    if (far.load()) return fail(LBM_ERR_CAPACITY, "neighbour tiles lie more than 2^30 values apart (tile plane too large)");

    lbm_tiling& I = T->info;
    I.ntx = ntx;
    I.nty = nty;
    I.ntz = ntz;
    I.n_tiles = (int32_t)n_tiles64;
    I.n_ftiles = count;
    I.nbr_per_tile = T->nn;
    I.n_fluid = n_fluid;
    I.pdf_bytes = (size_t)total * bpv;
    I.ghost_bytes = p->layout == LBM_LAYOUT_TGB ? 2 * (size_t)count * (size_t)tgb_ghost_per_tile(p->lattice, a) * bpv : 0;
    return LBM_OK;
}

// Several geometries in one tiling: each sample is tiled on its own and its
// tables are appended, with its tile indices (in the neighbour records) and
// its PDF offsets shifted past the samples before it.  The step kernels then
// treat the batch as one sparse geometry whose pieces never touch.
int build_batch_tiling(const lbm_params* p, int n, const int* dims, const uint8_t* const* masks, HostTiling* T,
                       std::vector<SampleRange>* samples) {
    if (!p || n < 1 || !dims || !masks) return fail(LBM_ERR_ARG, "batch: bad arguments");
    *T = HostTiling{};
    samples->clear();
    long long total_tiles = 0, total_values = 0, total_mesh = 0, total_fluid = 0;
    size_t total_bytes = 0, total_ghost = 0;
    for (int k = 0; k < n; k++) {
        lbm_params ps = *p;
        ps.nx = dims[3 * k];
        ps.ny = dims[3 * k + 1];
        ps.nz = dims[3 * k + 2];
        HostTiling S;
        int rc = build_tiling(&ps, masks[k], &S);
        if (rc) {
            char msg[400];
            snprintf(msg, sizeof msg, "%s", g_err);
            return fail(rc, "batch sample %d: %s", k, msg);
        }
        if (total_tiles + S.info.n_ftiles > INT32_MAX) return fail(LBM_ERR_CAPACITY, "batch: too many tiles");
        const int base_t = (int)total_tiles;
        T->a = S.a;
        T->d = S.d;
        T->nn = S.nn;
        T->words = S.words;
        T->tmask.insert(T->tmask.end(), S.tmask.begin(), S.tmask.end());
        T->coords.insert(T->coords.end(), S.coords.begin(), S.coords.end());
        for (int32_t v : S.nbr) T->nbr.push_back(v >= 0 ? v + base_t : -1);
        for (long long o : S.tile_off) T->tile_off.push_back(o + total_values);
        T->tile_stride.insert(T->tile_stride.end(), S.tile_stride.begin(), S.tile_stride.end());
        samples->push_back(SampleRange{ps.nx, ps.ny, ps.nz, base_t, S.info.n_ftiles, S.info.n_fluid});
        total_tiles += S.info.n_ftiles;
        total_mesh += S.info.n_tiles;
        total_fluid += S.info.n_fluid;
        total_bytes += S.info.pdf_bytes;
        total_ghost += S.info.ghost_bytes;
        total_values += (long long)(S.info.pdf_bytes / bytes_per_value(p->storage));
    }
    const int nt = T->d == 3 ? T->a * T->a * T->a : T->a * T->a;
    if (total_tiles * nt > (long long)UINT32_MAX) return fail(LBM_ERR_CAPACITY, "batch: too many tile slots");
    lbm_tiling& I = T->info;
    I.ntx = I.nty = I.ntz = 0;
    I.n_tiles = (int32_t)(total_mesh > INT32_MAX ? INT32_MAX : total_mesh);
    I.n_ftiles = (int32_t)total_tiles;
    I.nbr_per_tile = T->nn;
    I.n_fluid = total_fluid;
    I.pdf_bytes = total_bytes;
    I.ghost_bytes = total_ghost;
    return LBM_OK;
}

int work_threads_for(int lattice, int a) {
    const int nt = lattice == LBM_D2Q9 ? a * a : a * a * a;
    return nt > 256 ? nt : 256;
}

// Fluid nodes in tile-major, row order, cut into blocks of consecutive tiles
// holding at most `threads` nodes and `max_tiles` tiles.
long long build_work_list(HostTiling* T, int threads, int max_tiles, bool want_nodes, bool split_tiles) {
    const int nt = T->d == 3 ? T->a * T->a * T->a : T->a * T->a;
    const int32_t n = T->info.n_ftiles;
    T->nodes.clear();
    T->blocks.clear();
    // first node of every tile (a prefix count), then the block boundaries
    // (a tile's stride is its fluid count: the compact layout has no padding)
    const bool have_counts = T->tile_stride.size() == (size_t)n;
    std::vector<int64_t> first((size_t)n + 1, 0);
    for (int32_t k = 0; k < n; k++) {
        int nf = 0;
        if (have_counts) {
            nf = T->tile_stride[k];
        } else {
            const uint64_t* m = &T->tmask[(size_t)k * T->words];
            for (int w = 0; w < T->words; w++) nf += __builtin_popcountll(m[w]);
        }
        first[k + 1] = first[k] + nf;
    }
    WorkBlock cur{0, 0, 0, 0};
    if (split_tiles) {
        // every block full (`threads` nodes) but the last: a tile that does not
        // fit continues in the next block (the list holds a tile's nodes in a row)
        for (int32_t k = 0; k < n; k++) {
            int64_t at = first[k];
            while (at < first[k + 1]) {
                if (cur.n_tiles == max_tiles) {
                    T->blocks.push_back(cur);
                    cur = WorkBlock{0, 0, 0, 0};
                }
                if (cur.n_tiles == 0) {
                    cur.node_begin = (int)at;
                    cur.tile_begin = k;
                }
                const int take = (int)std::min<int64_t>(first[k + 1] - at, threads - cur.count);
                cur.count += take;
                cur.n_tiles++;
                at += take;
                if (cur.count == threads) {
                    T->blocks.push_back(cur);
                    cur = WorkBlock{0, 0, 0, 0};
                }
            }
        }
    } else {
        for (int32_t k = 0; k < n; k++) {
            const int nf = (int)(first[k + 1] - first[k]);
            if (cur.n_tiles > 0 && (cur.count + nf > threads || cur.n_tiles == max_tiles)) {
                T->blocks.push_back(cur);
                cur = WorkBlock{0, 0, 0, 0};
            }
            if (cur.n_tiles == 0) {
                cur.node_begin = (int)first[k];
                cur.tile_begin = k;
            }
            cur.count += nf;
            cur.n_tiles++;
        }
    }
    if (cur.n_tiles > 0) T->blocks.push_back(cur);
    if (!want_nodes) return first[n];
    // the nodes of each tile in row order, tiles in parallel
    T->nodes.resize((size_t)first[n]);
    parallel_ranges(n, 1024, [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; k++) {
            const uint64_t* m = &T->tmask[(size_t)k * T->words];
            uint32_t* out = &T->nodes[(size_t)first[k]];
            for (int node = 0; node < nt; node++)
                if ((m[node >> 6] >> (node & 63)) & 1ull) *out++ = (uint32_t)k * (uint32_t)nt + node;
        }
    });
    return first[n];
}

}  // namespace lbm

extern "C" int lbm_build_tilemap(const lbm_params* p, const uint8_t* mask, int32_t* tile_map,
                                 int32_t* nbr, lbm_tiling* out) {
    using namespace lbm;
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    HostTiling T;
    int rc = build_tiling(p, mask, &T, nbr != nullptr);  // a size query skips the neighbour records
    if (rc) return rc;
    *out = T.info;
    if (tile_map) std::memcpy(tile_map, T.tile_map.data(), T.tile_map.size() * sizeof(int32_t));
    if (nbr) std::memcpy(nbr, T.nbr.data(), T.nbr.size() * sizeof(int32_t));
    return LBM_OK;
}

extern "C" int lbm_build_tilemap_batch(const lbm_params* p, int n_samples, const int* dims,
                                       const uint8_t* const* masks, lbm_tiling* out) {
    using namespace lbm;
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    HostTiling T;
    std::vector<SampleRange> samples;
    int rc = build_batch_tiling(p, n_samples, dims, masks, &T, &samples);
    if (rc) return rc;
    *out = T.info;
    return LBM_OK;
}

extern "C" const char* lbm_last_error(void) { return lbm::g_err; }
