// Plan construction, drivers and the C ABI of include/fbs.h.
//
// Plan time (once per (N, L, edges)):
//   * integer thresholds on |m|^2 from the physical edges (the scalar reading
//     of the bin-width rule of Eq. gen_Nspec3);
//   * shell sizes |S_b| and the extreme |m|^2 of each shell, by enumerating
//     the lattice;
//   * candidate bin triples (and quadruples) that can close a polygon;
//   * the count fields N_b of Eq. delta_nr in FP64 on the device, and the
//     exact ordered counts N_tri = sum_n N_a N_b N_c / N_pix (the denominator
//     of Eq. gen_Nspec3), rounded to int64 and checked for integrality;
//   * the closed-triplet list and its pair-grouped work list.
// Per field: forward FFT -> inverse per shell -> real-space product sums ->
// FP64 normalisation (Eqs. Jeong_PS, Jeong_BI, Jeong_gen).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fbs_internal.h"
#include "levels.h"

namespace fbs {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    fbs_status st = (e == cudaErrorMemoryAllocation) ? FBS_ERR_OOM : FBS_ERR_CUDA;
    throw Failure{st, std::string(what) + ": " + cudaGetErrorString(e)};
}

FftFactors make_factors(int n) {
    FftFactors f{};
    f.n = n;
    int m = n, a = 0, b = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++b; }
    if (m != 1 || n > 4096) throw Failure{FBS_ERR_UNSUPPORTED_N, "length is not 2^a 3^b"};
    int k = 0;
    for (int i = 0; i < a / 3; ++i) f.r[k++] = 8;
    if (a % 3 == 1) f.r[k++] = 2;
    if (a % 3 == 2) f.r[k++] = 4;
    for (int i = 0; i < b; ++i) f.r[k++] = 3;
    f.nst = k;
    return f;
}

// ---------------------------------------------------------------- device budget
static std::atomic<long long> g_budget{0};   // 0: no budget
static std::atomic<long long> g_in_use{0};   // bytes held by all plans (and their transient buffers)

void budget_reserve(long long bytes) {
    const long long prev = g_in_use.fetch_add(bytes);
    const long long cap = g_budget.load();
    if (cap > 0 && prev + bytes > cap) {
        g_in_use.fetch_sub(bytes);
        throw Failure{FBS_ERR_OOM, "device budget: " + std::to_string(prev) + " + " + std::to_string(bytes) +
                                       " bytes exceeds " + std::to_string(cap)};
    }
}

void budget_release(long long bytes) { g_in_use.fetch_sub(bytes); }

AsyncBuf::AsyncBuf(size_t n, cudaStream_t s, const char *what) : stream(s) {
    if (n == 0) n = 16;
    budget_reserve((long long)n);
    if (cudaMallocAsync(&ptr, n, s) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        budget_release((long long)n);
        throw Failure{FBS_ERR_OOM, std::string(what) + ": device allocation failed"};
    }
    bytes = (long long)n;
}

AsyncBuf::~AsyncBuf() {
    if (ptr) {
        cudaFreeAsync(ptr, stream);
        cudaGetLastError();
        budget_release(bytes);
    }
}

void *Plan::dalloc(size_t bytes) {
    if (root_) return root_->dalloc(bytes);  // a level's memory belongs to its root
    void *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    budget_reserve((long long)bytes);
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        budget_release((long long)bytes);
        throw Failure{e == cudaErrorMemoryAllocation ? FBS_ERR_OOM : FBS_ERR_CUDA,
                      "cudaMalloc(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e)};
    }
    allocs.push_back(ptr);
    dev_bytes += (long long)bytes;
    return ptr;
}

// ---------------------------------------------------------------- timing
static constexpr size_t kMaxPending = 2048;

void Plan::tic(int cls, int &slot) {
    if (root_) {  // a level's launches are timed by its root
        root_->tic(cls, slot);
        return;
    }
    slot = -1;
    if (!(flags & FBS_FLAG_TIMING)) return;
    if (pending.size() >= kMaxPending) flush_times();
    const int idx = (int)pending.size();
    while (evs.size() < 2 * (size_t)(idx + 1)) {
        cudaEvent_t e;
        FBS_CUDA(cudaEventCreate(&e));
        evs.push_back(e);
    }
    FBS_CUDA(cudaEventRecord(evs[2 * idx], stream));
    pending.push_back({cls, idx});
    slot = idx;
}

void Plan::toc(int slot) {
    if (root_) {
        root_->toc(slot);
        return;
    }
    if (slot < 0) return;
    cudaEventRecord(evs[2 * slot + 1], stream);
}

void Plan::flush_times() {
    if (pending.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto &pr : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, evs[2 * pr.second], evs[2 * pr.second + 1]) == cudaSuccess) {
            kt_ms[pr.first] += ms;
            kt_n[pr.first] += 1;
        } else {
            cudaGetLastError();
        }
    }
    pending.clear();
}

// ---------------------------------------------------------------- plan helpers
// Smallest integer |m|^2 with |m| k_f >= edge: ceil((edge/k_f)^2), after
// snapping values within 1e-9 (relative) of an integer onto it so that edges
// at whole multiples of k_f land where they were meant to.
static long long edge_threshold(double edge, double L) {
    if (edge <= 0.0) return 0;
    const double kf = 2.0 * M_PI / L;
    const double q = edge / kf;
    double s = q * q;
    double r = nearbyint(s);
    if (fabs(s - r) <= 1e-9 * fmax(1.0, s)) s = r;
    return (long long)ceil(s);
}

static bool good_N(int N) {
    if (N < 8 || N > 512 || (N & 1)) return false;
    int m = N;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

static int isqrt_floor(long long v) {
    if (v <= 0) return 0;
    long long r = (long long)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return (int)r;
}

template <typename T>
static T *upload(Plan &p, const std::vector<T> &v) {
    T *d = (T *)p.dalloc(std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty())
        FBS_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, p.stream));
    return d;
}

static bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Shells: sizes and min/max |m|^2 by lattice enumeration over |m_j| <= Rmax
// with components in [-N/2, N/2).
static void enumerate_shells(Plan &p, std::vector<long long> &mn, std::vector<long long> &mx) {
    const int N = p.N, nb = p.nbins;
    const long long top = p.thr[nb];
    int Rmax = std::min(isqrt_floor(top - 1), N / 2);
    p.shell.assign(nb, 0);
    p.selfconj.assign(nb, 0);
    mn.assign(nb, -1);
    mx.assign(nb, -1);
    std::vector<int> lut;  // bin of each |m|^2 < top
    lut.assign((size_t)std::max<long long>(top, 1), -1);
    for (int b = 0; b < nb; ++b)
        for (long long s = p.thr[b]; s < p.thr[b + 1]; ++s) lut[s] = b;
    const int lo = -Rmax, hi = std::min(Rmax, N / 2 - 1);
    for (int x = lo; x <= hi; ++x)
        for (int y = lo; y <= hi; ++y) {
            long long r2 = (long long)x * x + (long long)y * y;
            if (r2 >= top) continue;
            for (int z = lo; z <= hi; ++z) {
                long long s = r2 + (long long)z * z;
                if (s >= top) continue;
                int b = lut[s];
                if (b < 0) continue;
                p.shell[b] += 1;
                // m = -m (mod N): every component 0 or -N/2
                if ((x == 0 || 2 * x == -N) && (y == 0 || 2 * y == -N) && (z == 0 || 2 * z == -N))
                    p.selfconj[b] += 1;
                if (mn[b] < 0 || s < mn[b]) mn[b] = s;
                if (s > mx[b]) mx[b] = s;
            }
        }
}

// Largest component |m_j| a mode of global bin b can have.
static int bin_R(const Plan &root, int b) { return std::min(isqrt_floor(root.thr[b + 1] - 1), root.N / 2); }

// Geometry of a level: its bins' boxes on the level's grid M.  The spectrum
// box (forward output, transform length N) is the root's.
static void build_level_geometry(Plan &root, Plan &lv) {
    const int M = lv.M;
    lv.nbins = (int)lv.gbin.size();
    lv.geom.assign(lv.nbins, BinGeom{});
    long long aoff = 0;
    for (int b = 0; b < lv.nbins; ++b) {
        const int gb = lv.gbin[b];
        BinGeom &g = lv.geom[b];
        g.thr_lo = root.thr[gb];
        g.thr_hi = root.thr[gb + 1];
        g.empty = 0;  // levels hold non-empty bins only
        g.Rb = std::min(isqrt_floor(g.thr_hi - 1), M / 2);
        g.Db = (2 * g.Rb + 1 > M) ? M : 2 * g.Rb + 1;
        g.Dzb = std::min(g.Rb, M / 2) + 1;
        g.A_off = aoff;
        aoff += (long long)M * g.Db * g.Dzb;
    }
    lv.A_elems = aoff;
    lv.box = root.box;
    lv.boxM = root.box;
    lv.boxM.N = M;
    long long gplane = 0;
    for (int b = 0; b < lv.nbins; ++b) gplane += (long long)M * lv.geom[b].Dzb;
    lv.G_plane = gplane;
}

static void set_slab_offsets(Plan &p) {
    long long goff = 0;
    for (int b = 0; b < p.nbins; ++b) {
        p.geom[b].G_off = goff;
        if (!p.geom[b].empty) goff += (long long)p.slab * p.M * p.geom[b].Dzb;
    }
}

// Candidate bin triples (a <= b <= c over non-empty bins).  Unless aliased
// closure is allowed, every component is below N/4, so closure modulo N is
// exact closure and needs |m_c| <= |m_a| + |m_b|: keep the triple when the
// smallest |m| of c does not exceed the largest |m| of a plus that of b.
static void candidates(const Plan &p, const std::vector<long long> &mn,
                       const std::vector<long long> &mx, int arity, std::vector<int> &items) {
    const int nb = p.nbins;
    const bool all = (p.flags & FBS_FLAG_ALLOW_ALIASED) != 0;
    items.clear();
    auto hi = [&](int b) { return sqrt((double)mx[b]); };
    auto lo = [&](int b) { return sqrt((double)mn[b]); };
    for (int a = 0; a < nb; ++a) {
        if (!p.shell[a]) continue;
        for (int b = a; b < nb; ++b) {
            if (!p.shell[b]) continue;
            for (int c = b; c < nb; ++c) {
                if (!p.shell[c]) continue;
                if (arity == 3) {
                    if (all || lo(c) <= hi(a) + hi(b) + 1e-9) {
                        items.push_back(a);
                        items.push_back(b);
                        items.push_back(c);
                    }
                } else {
                    for (int d = c; d < nb; ++d) {
                        if (!p.shell[d]) continue;
                        if (all || lo(d) <= hi(a) + hi(b) + hi(c) + 1e-9) {
                            items.push_back(a);
                            items.push_back(b);
                            items.push_back(c);
                            items.push_back(d);
                        }
                    }
                }
            }
        }
    }
}

// FP64 fields on the octant of the level's grid -- for every weight table
// (nullptr: the plain shell indicator, the count field N_b of Eq. delta_nr)
// and every bin of the level, row f * nbins + b.
static std::unique_ptr<AsyncBuf> octant_fields(Plan &p, const std::vector<const double *> &wtabs) {
    const int N = p.M, H = N / 2 + 1;  // the evaluation grid (exact for these products)
    const long long H3 = (long long)H * H * H;
    const int nb = p.nbins, nf = (int)wtabs.size();
    auto noct_buf = std::make_unique<AsyncBuf>((size_t)nf * nb * H3 * sizeof(double), p.stream, "octant fields");
    double *noct = noct_buf->as<double>();
    // bin groups bounded by ~2 GB of FP64 scratch
    const long long budget = 2LL << 30;
    for (int f = 0; f < nf; ++f) {
        int b0 = 0;
        while (b0 < nb) {
            long long a_el = 0, g_el = 0;
            int b1 = b0;
            std::vector<BinGeom> gg;
            while (b1 < nb) {
                const BinGeom &g = p.geom[b1];
                long long da = g.empty ? 0 : (long long)N * g.Db * g.Dzb;
                long long dg = g.empty ? 0 : (long long)H * N * g.Dzb;
                if (b1 > b0 && (a_el + da + g_el + dg) * 16 > budget) break;
                BinGeom q = g;
                q.A_off = a_el;
                q.G_off = g_el;
                gg.push_back(q);
                a_el += da;
                g_el += dg;
                ++b1;
            }
            {
                AsyncBuf A64(std::max<long long>(1, a_el) * 16, p.stream, "count scratch");
                AsyncBuf G64(std::max<long long>(1, g_el) * 16, p.stream, "count scratch");
                AsyncBuf dgeom(gg.size() * sizeof(BinGeom), p.stream, "count scratch");
                FBS_CUDA(cudaMemcpyAsync(dgeom.ptr, gg.data(), gg.size() * sizeof(BinGeom), cudaMemcpyHostToDevice,
                                         p.stream));
                launch_count_fields_fp64_impl(p, noct + ((long long)f * nb + b0) * H3, b0, b1 - b0,
                                              A64.as<double2>(), G64.as<double2>(), dgeom.as<BinGeom>(), wtabs[f]);
            }
            FBS_CUDA(cudaStreamSynchronize(p.stream));  // gg goes out of scope
            b0 = b1;
        }
    }
    return noct_buf;
}

// The octant sums of the products of the rows each item names (arity rows
// per item) of the octant fields noct (nrows rows).
static void octant_contract(Plan &p, const double *noct, int nrows, const std::vector<int> &items, int arity,
                            std::vector<double> &den) {
    const int n = (int)(items.size() / arity);
    den.assign(n, 0.0);
    if (n == 0) return;
    AsyncBuf items_buf(items.size() * sizeof(int), p.stream, "count items");
    AsyncBuf den_buf(n * sizeof(double), p.stream, "count items");
    FBS_CUDA(cudaMemcpyAsync(items_buf.ptr, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice,
                             p.stream));
    launch_count_contraction(p, noct, nrows, 0, items_buf.as<int>(), n, arity, den_buf.as<double>());
    FBS_CUDA(cudaMemcpyAsync(den.data(), den_buf.ptr, n * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
}

static void octant_sums(Plan &p, const std::vector<const double *> &wtabs, const std::vector<int> &items,
                        int arity, std::vector<double> &den) {
    den.assign(items.size() / arity, 0.0);
    if (items.empty()) return;
    auto f = octant_fields(p, wtabs);
    octant_contract(p, f->as<double>(), (int)wtabs.size() * p.nbins, items, arity, den);
}

// FP64 count fields on the octant, the count sums of all candidates, and the
// exact quadruple counts from the same fields.
static void exact_counts(Plan &p, const std::vector<int> &tc, const std::vector<int> &qc,
                         std::vector<double> &tden, std::vector<double> &qden, std::vector<U128> &qexact) {
    tden.assign(tc.size() / 3, 0.0);
    qden.assign(qc.size() / 4, 0.0);
    qexact.assign(qc.size() / 4, U128{});
    if (tc.empty() && qc.empty()) return;
    auto f = octant_fields(p, {nullptr});
    octant_contract(p, f->as<double>(), p.nbins, tc, 3, tden);
    octant_contract(p, f->as<double>(), p.nbins, qc, 4, qden);
    exact_quad_counts(p, f->as<double>(), qc, qexact);
}

static double u128_to_double(const U128 &v) {
    return (double)(((unsigned __int128)v.hi << 64) | v.lo);  // correctly rounded
}

// Round sum_n N..N / N_pix to the count.  The FP64 sum carries rounding
// error that grows with the count (about 1e-15 relative); a distance above
// 0.25 from the nearest integer means the rounding could be wrong.
static int64_t round_count(Plan &p, double den, double npix) {
    double v = den / npix;
    double r = nearbyint(v);
    double d = fabs(v - r);
    if (d > p.count_margin) p.count_margin = d;
    if (d > 0.25)
        throw Failure{FBS_ERR_NUMERIC, "count sum " + std::to_string(v) + " is not an integer"};
    return (int64_t)r;
}

static void build_tasks(Plan &p) {
    // bispectrum: outer pair (b, c), inner a; items sorted by (b, c, a)
    {
        const int nt = (int)p.ntri.size();
        std::vector<int> ord(nt);
        for (int i = 0; i < nt; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int u, int v) {
            const int32_t *x = &p.trip[3 * u], *y = &p.trip[3 * v];
            if (x[1] != y[1]) return x[1] < y[1];
            if (x[2] != y[2]) return x[2] < y[2];
            return x[0] < y[0];
        });
        TaskList &t = p.ttask;
        t = TaskList{};
        int lb = -1, lc = -1;
        for (int i : ord) {
            const int32_t *x = &p.trip[3 * i];
            if (x[1] != lb || x[2] != lc) {
                t.pb.push_back(x[1]);
                t.pc.push_back(x[2]);
                t.pstart.push_back((int)t.ia.size());
                lb = x[1];
                lc = x[2];
            }
            t.ia.push_back(x[0]);
            t.ib.push_back(-1);
            t.iout.push_back(i);
        }
        t.npairs = (int)t.pb.size();
        t.nitems = (int)t.ia.size();
        t.pstart.push_back(t.nitems);
    }
    // trispectrum: outer pair (c, d), inner (a, b)
    {
        const int nq = (int)p.nquad.size();
        std::vector<int> ord(nq);
        for (int i = 0; i < nq; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int u, int v) {
            const int32_t *x = &p.quad[4 * u], *y = &p.quad[4 * v];
            if (x[2] != y[2]) return x[2] < y[2];
            if (x[3] != y[3]) return x[3] < y[3];
            if (x[0] != y[0]) return x[0] < y[0];
            return x[1] < y[1];
        });
        TaskList &t = p.qtask;
        t = TaskList{};
        int lc = -1, ld = -1;
        for (int i : ord) {
            const int32_t *x = &p.quad[4 * i];
            if (x[2] != lc || x[3] != ld) {
                t.pb.push_back(x[2]);
                t.pc.push_back(x[3]);
                t.pstart.push_back((int)t.ia.size());
                lc = x[2];
                ld = x[3];
            }
            t.ia.push_back(x[0]);
            t.ib.push_back(x[1]);
            t.iout.push_back(i);
        }
        t.npairs = (int)t.pb.size();
        t.nitems = (int)t.ia.size();
        t.pstart.push_back(t.nitems);
    }
}

static std::atomic<long long> g_slab_default{0};  // 0: 8 GiB

static long long slab_budget_bytes() {
    const char *e = getenv("FBS_SLAB_MB");
    if (e && atoll(e) > 0) return atoll(e) << 20;
    const long long d = g_slab_default.load();
    return d > 0 ? d : 8LL << 30;
}

// ---------------------------------------------------------------- levels
// Smallest level grid of multi-level plans.  BF16x3 products carry ~2^-17
// relative rounding each; a level's sums average it over M^3 points, so the
// error of a cancelling item grows like (N/M)^(3/2) on smaller grids.  Over
// every triplet of 256^3 workloads (32 linear and 48 log bins, gated on the
// FP64 cancellation-free scale) the worst BF16x3 error was 1.1e-4 with
// levels down to M = 32 and 3.8e-5 with M >= 64, against the 2e-4 gate.
static constexpr int kMinLevelGrid = 64;

// Plan-time results carried over from an exported plan: the closed items
// (global bins, ascending) and their exact counts.
struct CountCache {
    std::map<std::array<int, 4>, double> counts;  // triplets (b[3] = -1)
    std::map<std::array<int, 4>, U128> qcounts;   // quadruplets
    double margin = 0;
};

// Serialised form (native byte order): "FBSC", version, N, flags, nbins,
// L, thr[nbins+1], ntrip, ntrip x (a, b, c, N_tri), nquad,
// nquad x (a, b, c, d, N_quad low 64 bits, N_quad high 64 bits), count margin.
static constexpr uint32_t kCacheMagic = 0x43534246u;  // "FBSC"
static constexpr uint32_t kCacheVersion = 2u;

struct Writer {
    std::vector<unsigned char> b;
    template <typename T> void put(const T &v) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
        b.insert(b.end(), p, p + sizeof(T));
    }
};

struct Reader {
    const unsigned char *p;
    size_t n, off = 0;
    template <typename T> T get() {
        if (off + sizeof(T) > n) throw Failure{FBS_ERR_ARG, "plan counts blob is truncated"};
        T v;
        memcpy(&v, p + off, sizeof(T));
        off += sizeof(T);
        return v;
    }
};

static std::vector<unsigned char> export_counts(const Plan &p) {
    Writer w;
    w.put(kCacheMagic);
    w.put(kCacheVersion);
    w.put((int32_t)p.N);
    w.put((uint32_t)(p.flags & (FBS_FLAG_TRISPECTRUM | FBS_FLAG_ALLOW_ALIASED)));
    w.put((int32_t)p.nbins);
    w.put(p.L);
    for (long long t : p.thr) w.put((int64_t)t);
    w.put((int64_t)p.ntri.size());
    for (size_t i = 0; i < p.ntri.size(); ++i) {
        for (int k = 0; k < 3; ++k) w.put((int32_t)p.trip[3 * i + k]);
        w.put((int64_t)p.ntri[i]);
    }
    w.put((int64_t)p.nquad.size());
    for (size_t i = 0; i < p.nquad.size(); ++i) {
        for (int k = 0; k < 4; ++k) w.put((int32_t)p.quad[4 * i + k]);
        w.put((uint64_t)p.nquad128[i].lo);
        w.put((uint64_t)p.nquad128[i].hi);
    }
    w.put(p.count_margin);
    return w.b;
}

// Parse a blob and check it describes this plan's bins (same N, L, flags
// that change the item set, and the same integer thresholds).
static void import_counts(const Plan &p, const void *blob, int64_t size, CountCache &c) {
    if (!blob || size <= 0) throw Failure{FBS_ERR_ARG, "empty plan counts blob"};
    Reader r{reinterpret_cast<const unsigned char *>(blob), (size_t)size};
    if (r.get<uint32_t>() != kCacheMagic || r.get<uint32_t>() != kCacheVersion)
        throw Failure{FBS_ERR_ARG, "not a plan counts blob of this library version"};
    const int N = r.get<int32_t>();
    const uint32_t fl = r.get<uint32_t>();
    const int nb = r.get<int32_t>();
    const double L = r.get<double>();
    if (N != p.N || nb != p.nbins || L != p.L ||
        fl != (p.flags & (FBS_FLAG_TRISPECTRUM | FBS_FLAG_ALLOW_ALIASED)))
        throw Failure{FBS_ERR_ARG, "plan counts blob is for another grid, box, bin count or flags"};
    for (int i = 0; i <= nb; ++i)
        if (r.get<int64_t>() != p.thr[i]) throw Failure{FBS_ERR_ARG, "plan counts blob is for other bin edges"};
    const int64_t nt = r.get<int64_t>();
    if (nt < 0) throw Failure{FBS_ERR_ARG, "bad plan counts blob"};
    for (int64_t i = 0; i < nt; ++i) {
        std::array<int, 4> k{r.get<int32_t>(), r.get<int32_t>(), r.get<int32_t>(), -1};
        c.counts[k] = (double)r.get<int64_t>();
    }
    const int64_t nq = r.get<int64_t>();
    if (nq < 0) throw Failure{FBS_ERR_ARG, "bad plan counts blob"};
    for (int64_t i = 0; i < nq; ++i) {
        std::array<int, 4> k{r.get<int32_t>(), r.get<int32_t>(), r.get<int32_t>(), r.get<int32_t>()};
        U128 v;
        v.lo = r.get<uint64_t>();
        v.hi = r.get<uint64_t>();
        c.qcounts[k] = v;
    }
    c.margin = r.get<double>();
}

static Plan *new_level(Plan &root, int M) {
    Plan *lv = new Plan();
    lv->root_ = &root;
    lv->N = root.N;
    lv->L = root.L;
    lv->M = M;
    lv->fM = make_factors(M);
    lv->precision = root.precision;
    lv->flags = root.flags;
    lv->stream = root.stream;
    lv->tc_wide = root.tc_wide;
    lv->tc_roles = root.tc_roles;
    lv->tc_chunk = root.tc_chunk;
    lv->tc_pairs = root.tc_pairs;
    lv->tc_merge = root.tc_merge;
    lv->tc_bstages = root.tc_bstages;
    lv->tc_bfroma = root.tc_bfroma;
    lv->tc_stack = root.tc_stack;
    lv->tc_wait_limit = root.tc_wait_limit;
    lv->d_box = root.d_box;
    root.levels.push_back(lv);
    return lv;
}

static void create_plan(Plan &p, const double *edges, const void *blob = nullptr, int64_t blob_size = 0) {
    const int N = p.N, nb = p.nbins;
    const bool quads_on = (p.flags & FBS_FLAG_TRISPECTRUM) != 0;
    p.fN = make_factors(N);
    p.thr.resize(nb + 1);
    for (int i = 0; i <= nb; ++i) p.thr[i] = edge_threshold(edges[i], p.L);
    for (int i = 0; i < nb; ++i)
        if (p.thr[i + 1] < p.thr[i]) throw Failure{FBS_ERR_ARG, "edges must be ascending"};
    if (!(p.flags & FBS_FLAG_ALLOW_ALIASED)) {
        // top edge <= N k_f / 4  <=>  thr[nb] <= (N/4)^2 (closure modulo N is exact closure)
        // ceil(N^2/16): |m|^2 < thr[nb] <= ceil(N^2/16) keeps every |m_j| < N/4
        const long long lim = ((long long)N * N + 15) / 16;
        if (p.thr[nb] > lim)
            throw Failure{FBS_ERR_ARG, "top edge beyond N k_f/4 (pass FBS_FLAG_ALLOW_ALIASED to allow)"};
    }
    std::unique_ptr<CountCache> cache;
    if (blob) {
        cache.reset(new CountCache());
        import_counts(p, blob, blob_size, *cache);
    }
    std::vector<long long> mn, mx;
    enumerate_shells(p, mn, mx);
    std::vector<int> R(nb, 0);
    int Rmax = 0;
    for (int b = 0; b < nb; ++b)
        if (p.shell[b]) {
            R[b] = bin_R(p, b);
            Rmax = std::max(Rmax, R[b]);
        }
    // the spectrum box of the forward transform: every mode of every bin
    p.box.N = N;
    p.box.R = Rmax;
    p.box.D = (2 * Rmax + 1 > N) ? N : 2 * Rmax + 1;
    p.box.Dz = std::min(Rmax, N / 2) + 1;
    p.M = N;

    // forward twiddles, spectrum box, timeout flags
    upload_forward_twiddles(p);
    p.d_box = (float2 *)p.dalloc((size_t)p.box.D * p.box.D * p.box.Dz * sizeof(float2));
    FBS_CUDA(cudaMemsetAsync(p.d_box, 0, (size_t)p.box.D * p.box.D * p.box.Dz * sizeof(float2), p.stream));
    p.d_errbuf = (int *)p.dalloc(2 * sizeof(int));
    FBS_CUDA(cudaMemsetAsync(p.d_errbuf, 0, 2 * sizeof(int), p.stream));

    // candidate items and the grid each needs
    std::vector<int> tc, qc;
    candidates(p, mn, mx, 3, tc);
    if (quads_on) candidates(p, mn, mx, 4, qc);
    std::vector<int> admissible;
    for (int M = 8; M <= N; ++M)
        if (good_N(M)) admissible.push_back(M);
    std::vector<LevelItem> items;
    const bool one_grid_N = (p.flags & (FBS_FLAG_FULL_GRID | FBS_FLAG_ALLOW_ALIASED)) != 0;
    const int single_M = one_grid_N ? N
                         : (p.flags & FBS_FLAG_SINGLE_GRID) ? grid_above(admissible, (quads_on ? 4 : 3) * Rmax, N)
                                                            : 0;
    for (int ar : {3, 4}) {
        const std::vector<int> &src = ar == 3 ? tc : qc;
        for (size_t i = 0; i < src.size() / ar; ++i) {
            LevelItem it{ar, {0, 0, 0, 0}, 0};
            int sum = 0, mxR = 0;
            for (int k = 0; k < ar; ++k) {
                it.b[k] = src[ar * i + k];
                sum += R[it.b[k]];
                mxR = std::max(mxR, R[it.b[k]]);
            }
            it.need = grid_above(admissible, std::max(sum, 2 * mxR), N);
            items.push_back(it);
        }
    }
    std::vector<int> Rb(nb, -1);
    for (int b = 0; b < nb; ++b)
        if (p.shell[b]) Rb[b] = R[b];
    // FBS_LEVEL_COST overrides the model's fixed cost per level (a negative
    // cost makes even small plans split into levels, as tests do)
    double per_level = 1e8;
    if (const char *e = getenv("FBS_LEVEL_COST")) per_level = atof(e);
    // the smallest level grid (FBS_MIN_LEVEL_GRID overrides): BF16 split
    // products carry ~2^-17 relative rounding each, so a level's sums must run
    // over enough points for it to average out on cancelling items
    int min_grid = kMinLevelGrid;
    if (const char *e = getenv("FBS_MIN_LEVEL_GRID")) min_grid = atoi(e);
    // (a single-grid plan keeps its documented grid M > pR)
    const LevelChoice lc = choose_levels(N, nb, Rb, items, single_M, fast_grids(), 4, per_level,
                                         single_M > 0 ? 0 : min_grid);
    const std::vector<int> &grids = lc.grids;
    for (int M : grids) new_level(p, M);
    std::vector<std::vector<int>> lt(grids.size()), lq(grids.size());  // candidate (global) items per level
    for (size_t i = 0; i < items.size(); ++i) {
        auto &dst = items[i].arity == 3 ? lt[lc.item_level[i]] : lq[lc.item_level[i]];
        dst.insert(dst.end(), items[i].b, items[i].b + items[i].arity);
    }

    // per level: geometry, twiddles, FP64 count fields and exact counts
    struct Closed {
        int level, local;  // index in the level's candidate list
    };
    std::vector<std::array<int, 4>> ctrip, cquad;   // closed items (global bins)
    std::vector<int64_t> ctri_cnt;
    std::vector<double> cquad_cnt;
    std::vector<U128> cquad_ex;
    std::vector<Closed> ctrip_src, cquad_src;
    std::vector<std::vector<int>> loc_of(grids.size());
    for (size_t l = 0; l < grids.size(); ++l) {
        Plan &lv = *p.levels[l];
        loc_of[l].assign(nb, -1);
        for (int b : lc.bins[l]) {
            loc_of[l][b] = (int)lv.gbin.size();
            lv.gbin.push_back(b);
        }
        build_level_geometry(p, lv);
        upload_eval_twiddles(lv);
        std::vector<int> ltc, lqc;
        for (int v : lt[l]) ltc.push_back(loc_of[l][v]);
        for (int v : lq[l]) lqc.push_back(loc_of[l][v]);
        std::vector<double> tden, qden;
        std::vector<U128> qex;
        // sum_M N_a N_b N_c / M^3 is the same integer as sum_N N_a N_b N_c / N^3
        const double npix = (double)lv.M * lv.M * lv.M;
        if (cache) {
            // counts carried over: the closed items and their exact counts, no count pass
            tden.assign(ltc.size() / 3, 0.0);
            qden.assign(lqc.size() / 4, 0.0);
            qex.assign(lqc.size() / 4, U128{});
            for (size_t i = 0; i < tden.size(); ++i) {
                auto it = cache->counts.find({lt[l][3 * i], lt[l][3 * i + 1], lt[l][3 * i + 2], -1});
                if (it != cache->counts.end()) tden[i] = it->second * npix;
            }
            for (size_t i = 0; i < qden.size(); ++i) {
                auto it = cache->qcounts.find({lq[l][4 * i], lq[l][4 * i + 1], lq[l][4 * i + 2], lq[l][4 * i + 3]});
                if (it != cache->qcounts.end()) {
                    qex[i] = it->second;
                    qden[i] = u128_to_double(it->second) * npix;
                }
            }
        } else {
            exact_counts(lv, ltc, lqc, tden, qden, qex);
        }
        for (size_t i = 0; i < tden.size(); ++i) {
            int64_t c = round_count(p, tden[i], npix);
            if (c < 0) throw Failure{FBS_ERR_NUMERIC, "negative triangle count"};
            if (c == 0) continue;
            ctrip.push_back({lt[l][3 * i], lt[l][3 * i + 1], lt[l][3 * i + 2], -1});
            ctri_cnt.push_back(c);
            ctrip_src.push_back({(int)l, (int)i});
        }
        for (size_t i = 0; i < qden.size(); ++i) {
            // Quadruple counts of wide shells reach 1e19 and more, past the exact
            // integers of FP64 (2^53) and of int64: the exact 128-bit counts
            // decide, the FP64 count-field sums only cross-check them
            const double c = u128_to_double(qex[i]);
            const double v = qden[i] / npix;
            if (!(fabs(v - c) <= 1e-6 * c + 0.5))
                throw Failure{FBS_ERR_NUMERIC, "exact and FP64 quadruple counts disagree (" + std::to_string(c) +
                                                   " vs " + std::to_string(v) + ")"};
            if (qex[i].lo == 0 && qex[i].hi == 0) continue;
            cquad.push_back({lq[l][4 * i], lq[l][4 * i + 1], lq[l][4 * i + 2], lq[l][4 * i + 3]});
            cquad_cnt.push_back(c);
            cquad_ex.push_back(qex[i]);
            cquad_src.push_back({(int)l, (int)i});
        }
    }
    if (cache) {
        if (ctrip.size() != cache->counts.size() || cquad.size() != cache->qcounts.size())
            throw Failure{FBS_ERR_ARG, "plan counts blob does not match this plan's candidate items"};
        p.count_margin = cache->margin;
    }
    // global output order: lexicographic over all levels
    std::vector<int> ot(ctrip.size()), oq(cquad.size());
    for (size_t i = 0; i < ot.size(); ++i) ot[i] = (int)i;
    for (size_t i = 0; i < oq.size(); ++i) oq[i] = (int)i;
    std::sort(ot.begin(), ot.end(), [&](int u, int v) { return ctrip[u] < ctrip[v]; });
    std::sort(oq.begin(), oq.end(), [&](int u, int v) { return cquad[u] < cquad[v]; });
    p.trip.clear();
    p.ntri.clear();
    p.quad.clear();
    p.nquad.clear();
    p.nquad128.clear();
    for (size_t g = 0; g < ot.size(); ++g) {
        const int i = ot[g];
        p.trip.insert(p.trip.end(), {ctrip[i][0], ctrip[i][1], ctrip[i][2]});
        p.ntri.push_back(ctri_cnt[i]);
        Plan &lv = *p.levels[ctrip_src[i].level];
        const auto &lo = loc_of[ctrip_src[i].level];
        lv.trip.insert(lv.trip.end(), {lo[ctrip[i][0]], lo[ctrip[i][1]], lo[ctrip[i][2]]});
        lv.ntri.push_back(ctri_cnt[i]);
        lv.gtrip.push_back((int)g);
    }
    for (size_t g = 0; g < oq.size(); ++g) {
        const int i = oq[g];
        p.quad.insert(p.quad.end(), {cquad[i][0], cquad[i][1], cquad[i][2], cquad[i][3]});
        p.nquad.push_back(cquad_cnt[i]);
        p.nquad128.push_back(cquad_ex[i]);
        Plan &lv = *p.levels[cquad_src[i].level];
        const auto &lo = loc_of[cquad_src[i].level];
        lv.quad.insert(lv.quad.end(), {lo[cquad[i][0]], lo[cquad[i][1]], lo[cquad[i][2]], lo[cquad[i][3]]});
        lv.nquad.push_back(cquad_cnt[i]);
        lv.gquad.push_back((int)g);
    }

    // per level: tasks, slabs, buffers.  The per-slab stages of the levels run
    // one after another on the plan's stream, so they share one set of
    // scratch buffers sized for the largest level.
    long long maxA = 1, maxG = 1, maxI = 1;
    for (size_t l = 0; l < grids.size(); ++l) {
        Plan &lv = *p.levels[l];
        build_tasks(lv);
        lv.tgrp = item_groups(lv.ttask, 8192);
        lv.qgrp = item_groups(lv.qtask, 8192);
        const int M = lv.M, lnb = lv.nbins;
        const long long per_plane = (long long)lnb * M * M * 4 + lv.G_plane * 8;
        const long long budget = slab_budget_bytes();
        int slab = (int)std::max<long long>(1, std::min<long long>(M, budget / std::max<long long>(1, per_plane)));
        const int nslabs = (M + slab - 1) / slab;
        slab = (M + nslabs - 1) / nslabs;  // balance the slabs
        lv.slab = slab;
        lv.slab_planned = slab;
        lv.nslabs = nslabs;
        set_slab_offsets(lv);
        maxA = std::max(maxA, lv.A_elems);
        maxG = std::max(maxG, lv.G_plane * lv.slab);
        maxI = std::max(maxI, (long long)lnb * lv.slab * M * M);
        lv.pbin.assign(lnb, -1);
        for (int b = 0; b < lnb; ++b)
            if (lc.bin_level[lv.gbin[b]] == (int)l) lv.pbin[b] = lv.gbin[b];
    }
    float2 *sA = (float2 *)p.dalloc((size_t)maxA * sizeof(float2));
    float2 *sG = (float2 *)p.dalloc((size_t)maxG * sizeof(float2));
    float *sI = (float *)p.dalloc((size_t)maxI * sizeof(float));
    p.part_blocks = contract_blocks();
    for (Plan *lp : p.levels) {
        Plan &lv = *lp;
        lv.d_box = p.d_box;
        lv.d_A = sA;
        lv.d_G = sG;
        lv.d_I = sI;
        lv.d_geom = upload(lv, lv.geom);
        lv.d_tpb = upload(lv, lv.ttask.pb);
        lv.d_tpc = upload(lv, lv.ttask.pc);
        lv.d_tps = upload(lv, lv.ttask.pstart);
        lv.d_tia = upload(lv, lv.ttask.ia);
        lv.d_tout = upload(lv, lv.ttask.iout);
        lv.d_tgrp = upload(lv, lv.tgrp);
        lv.d_qpb = upload(lv, lv.qtask.pb);
        lv.d_qpc = upload(lv, lv.qtask.pc);
        lv.d_qps = upload(lv, lv.qtask.pstart);
        lv.d_qia = upload(lv, lv.qtask.ia);
        lv.d_qib = upload(lv, lv.qtask.ib);
        lv.d_qout = upload(lv, lv.qtask.iout);
        lv.d_qgrp = upload(lv, lv.qgrp);
        lv.d_gtrip = upload(lv, lv.gtrip);
        lv.d_gquad = upload(lv, lv.gquad);
        lv.d_pbin = upload(lv, lv.pbin);
        const int ntl = (int)lv.ntri.size(), nql = (int)lv.nquad.size();
        lv.part_blocks = p.part_blocks;
        lv.d_tpart = (double *)lv.dalloc((size_t)lv.part_blocks * std::max(1, ntl) * sizeof(double));
        lv.d_qpart = (double *)lv.dalloc((size_t)lv.part_blocks * std::max(1, nql) * sizeof(double));
        lv.d_sumsq_part = (double *)lv.dalloc((size_t)lv.nbins * lv.M * zstage_row_groups(lv.M) * sizeof(double));
    }
    // the largest level stands for the plan in the single-grid queries
    int top = 0;
    for (size_t l = 1; l < grids.size(); ++l) top = (int)l;
    p.M = p.levels.empty() ? N : p.levels[top]->M;
    p.slab = p.levels.empty() ? 0 : p.levels[top]->slab;
    p.nslabs = p.levels.empty() ? 0 : p.levels[top]->nslabs;

    // per-field buffers of the root
    p.d_field = (float *)p.dalloc((size_t)N * N * N * sizeof(float));
    FBS_CUDA(cudaStreamCreateWithFlags(&p.copy_stream, cudaStreamNonBlocking));
    FBS_CUDA(cudaEventCreateWithFlags(&p.ev_field_ready, cudaEventDisableTiming));
    FBS_CUDA(cudaEventCreateWithFlags(&p.ev_field_free, cudaEventDisableTiming));
    FBS_CUDA(cudaEventCreateWithFlags(&p.ev_err, cudaEventDisableTiming));
    FBS_CUDA(cudaHostAlloc((void **)&p.h_err, sizeof(int), cudaHostAllocDefault));
    *p.h_err = 0;
    p.d_zbuf = (float2 *)p.dalloc((size_t)N * N * p.box.Dz * sizeof(float2));
    p.d_ybuf = (float2 *)p.dalloc((size_t)N * p.box.D * p.box.Dz * sizeof(float2));
    const int ntrip = (int)p.ntri.size(), nquad = (int)p.nquad.size();
    p.d_sumsq = (double *)p.dalloc(nb * sizeof(double));
    p.d_tnum = (double *)p.dalloc(std::max(1, ntrip) * sizeof(double));
    p.d_qnum = (double *)p.dalloc(std::max(1, nquad) * sizeof(double));
    p.d_B = (double *)p.dalloc(std::max(1, ntrip) * sizeof(double));
    p.d_T = (double *)p.dalloc(std::max(1, nquad) * sizeof(double));
    p.d_P = (double *)p.dalloc(nb * sizeof(double));
    p.d_ntri = upload(p, p.ntri);
    p.d_nquad = upload(p, p.nquad);
    p.d_shell = upload(p, p.shell);
    // every bin on the input grid (the shell moments of the spectrum box)
    p.geom.assign(nb, BinGeom{});
    for (int b = 0; b < nb; ++b) {
        BinGeom &g = p.geom[b];
        g.thr_lo = p.thr[b];
        g.thr_hi = p.thr[b + 1];
        g.empty = p.shell[b] == 0;
        g.Rb = g.empty ? 0 : bin_R(p, b);
        g.Db = (2 * g.Rb + 1 > N) ? N : 2 * g.Rb + 1;
        g.Dzb = std::min(g.Rb, N / 2) + 1;
    }
    p.d_geom = upload(p, p.geom);
    // unpaired quadruple counts of the connected trispectrum: N_quad minus the
    // paired ones (a = b < c = d: |S_a||S_c|; a = b = c = d: 3|S|^2 - 3|S| + Z)
    // (exact in 128-bit integers, then the nearest double)
    p.nconn.assign(nquad, 0.0);
    for (int i = 0; i < nquad; ++i) {
        const int32_t *q = &p.quad[4 * i];
        unsigned __int128 c = 0;
        if (q[0] == q[1] && q[2] == q[3]) {
            const unsigned __int128 sa = (unsigned long long)p.shell[q[0]], sc = (unsigned long long)p.shell[q[2]];
            c = q[0] != q[2] ? sa * sc : 3 * sa * sa - 3 * sa + (unsigned long long)p.selfconj[q[0]];
        }
        const unsigned __int128 t = ((unsigned __int128)p.nquad128[i].hi << 64) | p.nquad128[i].lo;
        if (c > t) throw Failure{FBS_ERR_NUMERIC, "paired quadruples exceed the quadruple count"};
        p.nconn[i] = (double)(t - c);
    }
    if (nquad > 0) {
        p.d_nconn = upload(p, p.nconn);
        p.d_quadtab = upload(p, p.quad);
        p.d_Tc = (double *)p.dalloc((size_t)nquad * sizeof(double));
    }
    p.d_mom_part = (double *)p.dalloc((size_t)nb * 16 * 3 * sizeof(double));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
}

// A host field is copied into the plan's staging buffer on the plan's own
// copy stream: it need not wait for kernels already queued on the plan's
// stream (another plan's evaluation, say), only for the previous forward
// transform to be done with the buffer.  Returns the device field.
static const float *stage_field(Plan &p, const float *field, bool &staged) {
    staged = !is_device_ptr(field);
    if (!staged) return field;
    const int N = p.N;
    if (p.field_free_recorded) FBS_CUDA(cudaStreamWaitEvent(p.copy_stream, p.ev_field_free, 0));
    FBS_CUDA(cudaMemcpyAsync(p.d_field, field, (size_t)N * N * N * sizeof(float), cudaMemcpyDefault, p.copy_stream));
    FBS_CUDA(cudaEventRecord(p.ev_field_ready, p.copy_stream));
    FBS_CUDA(cudaStreamWaitEvent(p.stream, p.ev_field_ready, 0));
    return p.d_field;
}

// After the forward transform has read a staged field.
static void release_field(Plan &p, bool staged) {
    if (!staged) return;
    FBS_CUDA(cudaEventRecord(p.ev_field_free, p.stream));
    p.field_free_recorded = true;
}

// The spectrum box of this evaluation: the field's forward transform, or a
// followed plan's box (field NULL) as its last evaluation on the shared
// stream left it.
static void forward_or_follow(Plan &p, const float *field) {
    if (p.leader) {
        if (field) throw Failure{FBS_ERR_STATE, "a following plan evaluates its leader's field: pass NULL"};
        if (p.leader->stream != p.stream)
            throw Failure{FBS_ERR_STATE, "a following plan must share its leader's stream"};
        return;
    }
    if (!field) throw Failure{FBS_ERR_ARG, "field is NULL"};
    bool staged = false;
    const float *d_in = stage_field(p, field, staged);
    launch_forward(p, d_in, nullptr, 1, p.d_zbuf, p.d_ybuf, p.d_box);
    release_field(p, staged);
}

static void run_field(Plan &p, const float *field, bool quads) {
    const bool tc = p.precision != FBS_PREC_FP32;
    if (tc) FBS_CUDA(cudaMemsetAsync(p.d_errbuf, 0, sizeof(int), p.stream));
    forward_or_follow(p, field);
    for (Plan *lp : p.levels) {
        Plan &lv = *lp;
        lv.fused_active = quads && tc && tc_fused_usable(lv);
        zero_partials(lv, quads);
        launch_inverse_x(lv, false);
        const int M = lv.M;
        const long long plane = (long long)M * M;
        for (int s = 0; s < lv.nslabs; ++s) {
            const int x0 = s * lv.slab;
            const int nx = std::min(lv.slab, M - x0);
            if (nx <= 0) break;
            launch_inverse_yz_slab(lv, x0, nx, lv.d_I);
            const long long npts = (long long)nx * plane;
            const long long stride = (long long)lv.slab * plane;
            if (lv.fused_active) {
                launch_contract_tc_fused(lv, lv.d_I, npts, stride);
                continue;
            }
            if (tc)
                launch_contract_tc(lv, lv.d_I, npts, stride, false);
            else
                launch_contract_fp32(lv, lv.d_I, npts, stride, false);
            if (quads) {
                // quadruplets on the tensor cores when the inner pairs fit one MMA (N <= 256)
                if (tc && tc_quads_usable(lv))
                    launch_contract_tc(lv, lv.d_I, npts, stride, true);
                else
                    launch_contract_fp32(lv, lv.d_I, npts, stride, true);
            }
        }
        launch_level_reduce(lv, quads);
    }
    launch_normalise(p, quads);
}

// ---------------------------------------------------------------- batches
// Buffers of batched evaluations (fbs_bispectrum_batch): every field of a
// batch gets its own forward scratch and spectrum box, and every level
// evaluates (field, bin) pairs as "virtual bins": bin b of field f is entry
// f * nbins + b of a geometry table whose offsets point into the field's own
// box, x-stage, y-stage and shell-field blocks.  The contraction and the
// reductions take the field from a grid dimension.
struct BatchLevel {
    BinGeom *d_vgeom = nullptr;
    int slab = 0, nslabs = 0;
    double *tpart = nullptr, *sq = nullptr;
};

struct BatchState {
    int cap = 0;
    float2 *zbuf = nullptr, *ybuf = nullptr, *box = nullptr, *A = nullptr, *G = nullptr;
    float *I = nullptr;
    double *tnum = nullptr, *sumsq = nullptr, *B = nullptr, *P = nullptr;
    const float **d_fptrs = nullptr;
    std::vector<const float *> ptrs;  // the pointer list last uploaded
    std::vector<BatchLevel> lv;
};

static BatchState &ensure_batch(Plan &p, int nf) {
    if (!p.batch) p.batch = new BatchState();
    BatchState &bs = *reinterpret_cast<BatchState *>(p.batch);
    if (bs.cap >= nf) return bs;
    // (re)allocate for nf fields; buffers of a smaller earlier batch stay with the plan
    const int N = p.N, D = p.box.D, Dz = p.box.Dz;
    const long long box_el = (long long)D * D * Dz;
    bs.zbuf = (float2 *)p.dalloc((size_t)nf * N * N * Dz * sizeof(float2));
    bs.ybuf = (float2 *)p.dalloc((size_t)nf * N * D * Dz * sizeof(float2));
    bs.box = (float2 *)p.dalloc((size_t)nf * box_el * sizeof(float2));
    FBS_CUDA(cudaMemsetAsync(bs.box, 0, (size_t)nf * box_el * sizeof(float2), p.stream));
    const size_t ntrip = std::max<size_t>(1, p.ntri.size());
    bs.tnum = (double *)p.dalloc((size_t)nf * ntrip * sizeof(double));
    bs.B = (double *)p.dalloc((size_t)nf * ntrip * sizeof(double));
    bs.sumsq = (double *)p.dalloc((size_t)nf * p.nbins * sizeof(double));
    bs.P = (double *)p.dalloc((size_t)nf * p.nbins * sizeof(double));
    bs.d_fptrs = (const float **)p.dalloc((size_t)nf * sizeof(float *));
    bs.ptrs.clear();
    long long maxA = 1, maxG = 1, maxI = 1;
    bs.lv.assign(p.levels.size(), BatchLevel{});
    const long long budget = slab_budget_bytes();
    for (size_t l = 0; l < p.levels.size(); ++l) {
        Plan &lv = *p.levels[l];
        BatchLevel &bl = bs.lv[l];
        const int M = lv.M, nb = lv.nbins;
        const long long per_plane = ((long long)nb * M * M * 4 + lv.G_plane * 8) * nf;
        int slab = (int)std::max<long long>(1, std::min<long long>(lv.slab_planned,
                                                                   budget / std::max<long long>(1, per_plane)));
        bl.nslabs = (M + slab - 1) / slab;
        bl.slab = (M + bl.nslabs - 1) / bl.nslabs;
        std::vector<BinGeom> vg((size_t)nf * nb);
        const long long gfield = lv.G_plane * bl.slab;
        for (int f = 0; f < nf; ++f) {
            long long goff = 0;
            for (int b = 0; b < nb; ++b) {
                BinGeom g = lv.geom[b];
                g.A_off += (long long)f * lv.A_elems;
                g.G_off = (long long)f * gfield + goff;
                g.box_off = (long long)f * box_el;
                goff += (long long)bl.slab * M * lv.geom[b].Dzb;
                vg[(size_t)f * nb + b] = g;
            }
        }
        bl.d_vgeom = upload(p, vg);
        bl.tpart = (double *)p.dalloc((size_t)nf * lv.part_blocks * std::max<size_t>(1, lv.ntri.size()) *
                                      sizeof(double));
        bl.sq = (double *)p.dalloc((size_t)nf * nb * M * zstage_row_groups(M) * sizeof(double));
        maxA = std::max(maxA, (long long)nf * lv.A_elems);
        maxG = std::max(maxG, nf * gfield);
        maxI = std::max(maxI, (long long)nf * nb * bl.slab * M * M);
    }
    bs.A = (float2 *)p.dalloc((size_t)maxA * sizeof(float2));
    bs.G = (float2 *)p.dalloc((size_t)maxG * sizeof(float2));
    bs.I = (float *)p.dalloc((size_t)maxI * sizeof(float));
    FBS_CUDA(cudaStreamSynchronize(p.stream));  // the host geometry tables go out of scope
    bs.cap = nf;
    return bs;
}

static void free_batch(Plan &p) {
    delete reinterpret_cast<BatchState *>(p.batch);  // device buffers belong to the plan's allocation list
    p.batch = nullptr;
}

static void run_batch(Plan &p, const float *const *fields, int nf) {
    BatchState &bs = ensure_batch(p, nf);
    std::vector<const float *> ptrs(fields, fields + nf);
    if (ptrs != bs.ptrs) {  // upload the pointer list only when it changes
        FBS_CUDA(cudaMemcpyAsync(bs.d_fptrs, ptrs.data(), nf * sizeof(float *), cudaMemcpyHostToDevice, p.stream));
        FBS_CUDA(cudaStreamSynchronize(p.stream));
        bs.ptrs = ptrs;
    }
    const bool tc = p.precision != FBS_PREC_FP32;
    if (tc) FBS_CUDA(cudaMemsetAsync(p.d_errbuf, 0, sizeof(int), p.stream));
    launch_forward(p, nullptr, bs.d_fptrs, nf, bs.zbuf, bs.ybuf, bs.box);
    for (size_t l = 0; l < p.levels.size(); ++l) {
        Plan &lv = *p.levels[l];
        const BatchLevel &bl = bs.lv[l];
        // the level's stages on the batch buffers and slabs, then back (the x
        // stage reads field f's spectrum at bs.box + f * box elements)
        float2 *A0 = lv.d_A, *G0 = lv.d_G, *box0 = lv.d_box;
        const int slab0 = lv.slab, nslabs0 = lv.nslabs;
        lv.d_A = bs.A;
        lv.d_G = bs.G;
        lv.d_box = bs.box;
        lv.slab = bl.slab;
        lv.nslabs = bl.nslabs;
        lv.fused_active = false;
        try {
            const int M = lv.M, nb = lv.nbins;
            FBS_CUDA(cudaMemsetAsync(bl.tpart, 0, (size_t)nf * lv.part_blocks * std::max<size_t>(1, lv.ntri.size()) *
                                                      sizeof(double), p.stream));
            FBS_CUDA(cudaMemsetAsync(bl.sq, 0, (size_t)nf * nb * M * zstage_row_groups(M) * sizeof(double),
                                     p.stream));
            launch_inverse_x_geom(lv, bl.d_vgeom, nb, nf * nb);
            const long long plane = (long long)M * M;
            for (int s = 0; s < bl.nslabs; ++s) {
                const int x0 = s * bl.slab;
                const int nx = std::min(bl.slab, M - x0);
                if (nx <= 0) break;
                launch_inverse_yz_slab_geom(lv, x0, nx, bs.I, bl.d_vgeom, nb, nf * nb, bl.sq);
                const long long npts = (long long)nx * plane, stride = (long long)bl.slab * plane;
                if (tc)
                    launch_contract_tc(lv, bs.I, npts, stride, false, nf, bl.tpart);
                else
                    launch_contract_fp32(lv, bs.I, npts, stride, false, nf, bl.tpart);
            }
            launch_level_reduce_batch(lv, false, nf, bl.tpart, bl.sq, bs.tnum, bs.sumsq);
        } catch (...) {
            lv.d_A = A0;
            lv.d_G = G0;
            lv.d_box = box0;
            lv.slab = slab0;
            lv.nslabs = nslabs0;
            throw;
        }
        lv.d_A = A0;
        lv.d_G = G0;
        lv.d_box = box0;
        lv.slab = slab0;
        lv.nslabs = nslabs0;
    }
    launch_normalise_batch(p, false, nf, bs.tnum, bs.sumsq, bs.B, bs.P);
}

// ---------------------------------------------------------------- diagonal-resolved trispectrum
// Per level: the pair-spectrum box (|q_j| <= Rq on the level grid), the
// half-box modes of every diagonal shell, a geometry whose y-stage offsets
// hold the whole grid in one slab, and the distinct pairs of the level's
// quadruplets (split (a, b) | (c, d)).
struct DiagLevel {
    BoxGeom bx{};
    int *d_idx = nullptr, *d_dstart = nullptr;
    float *d_w = nullptr;
    BinGeom *d_geom_full = nullptr;
    long long G_full = 0;
    std::vector<std::pair<int, int>> pairs;
    std::vector<std::array<int, 2>> qp;
};

struct DiagState {
    int nd = 0;
    std::vector<long long> thr;  // nd+1 thresholds on |q|^2
    std::vector<U128> cnt128;    // [nquad][nd] exact counts, plan order
    std::vector<double> cnt;
    double *d_cnt = nullptr, *d_num = nullptr, *d_TD = nullptr;
    std::vector<DiagLevel> lv;
};

static void free_diag(Plan &p) {
    delete reinterpret_cast<DiagState *>(p.diag);  // device buffers belong to the plan's allocation list
    p.diag = nullptr;
}

static void set_diagonal(Plan &p, const double *edges, int nd) {
    std::vector<long long> thr(nd + 1);
    for (int i = 0; i <= nd; ++i) {
        if (!(edges[i] >= 0.0) || (i > 0 && !(edges[i] > edges[i - 1])))
            throw Failure{FBS_ERR_ARG, "diagonal edges must be non-negative and ascending"};
        thr[i] = edges[i] > 0.0 ? edge_threshold(edges[i], p.L) : 0;
    }
    free_diag(p);
    DiagState *ds = new DiagState();
    p.diag = ds;
    ds->nd = nd;
    ds->thr = thr;
    const int nq = (int)p.nquad.size();
    ds->cnt128.assign((size_t)nq * nd, U128{});
    ds->lv.assign(p.levels.size(), DiagLevel{});
    for (size_t l = 0; l < p.levels.size(); ++l) {
        Plan &lv = *p.levels[l];
        DiagLevel &dl = ds->lv[l];
        const int nql = (int)lv.nquad.size();
        if (nql == 0) continue;
        const int M = lv.M;
        {
            // exact counts split by diagonal shell, from the level's count fields
            auto f = octant_fields(lv, {nullptr});
            std::vector<int> items(lv.quad.begin(), lv.quad.end());
            std::vector<U128> tot, dc;
            exact_quad_counts(lv, f->as<double>(), items, tot, &thr, &dc);
            for (int i = 0; i < nql; ++i)
                for (int D = 0; D < nd; ++D) ds->cnt128[(size_t)lv.gquad[i] * nd + D] = dc[(size_t)i * nd + D];
        }
        const long long top = thr[nd];
        int Rq = 0;
        while ((long long)(Rq + 1) * (Rq + 1) <= top - 1) ++Rq;
        Rq = std::min(Rq, M / 2);
        dl.bx.N = M;
        dl.bx.R = Rq;
        dl.bx.D = 2 * Rq + 1 > M ? M : 2 * Rq + 1;
        dl.bx.Dz = std::min(Rq, M / 2) + 1;
        std::vector<std::vector<int>> li(nd);
        std::vector<std::vector<float>> lw(nd);
        for (int jx = 0; jx < dl.bx.D; ++jx)
            for (int jy = 0; jy < dl.bx.D; ++jy)
                for (int jz = 0; jz < dl.bx.Dz; ++jz) {
                    const long long qx = box_freq(jx, dl.bx.D, M), qy = box_freq(jy, dl.bx.D, M);
                    const long long s2 = qx * qx + qy * qy + (long long)jz * jz;
                    if (s2 < thr[0] || s2 >= top) continue;
                    const int D = (int)(std::upper_bound(thr.begin(), thr.end(), s2) - thr.begin()) - 1;
                    li[D].push_back((int)(((long long)jx * dl.bx.D + jy) * dl.bx.Dz + jz));
                    lw[D].push_back(jz == 0 || 2 * jz == M ? 1.f : 2.f);
                }
        std::vector<int> idx, start(1, 0);
        std::vector<float> w;
        for (int D = 0; D < nd; ++D) {
            idx.insert(idx.end(), li[D].begin(), li[D].end());
            w.insert(w.end(), lw[D].begin(), lw[D].end());
            start.push_back((int)idx.size());
        }
        dl.d_idx = upload(lv, idx);
        dl.d_w = upload(lv, w);
        dl.d_dstart = upload(lv, start);
        std::vector<BinGeom> g = lv.geom;
        long long goff = 0;
        for (int b = 0; b < lv.nbins; ++b) {
            g[b].G_off = goff;
            if (!g[b].empty) goff += (long long)M * M * g[b].Dzb;
        }
        dl.G_full = std::max<long long>(1, goff);
        dl.d_geom_full = upload(lv, g);
        std::map<std::pair<int, int>, int> pid;
        dl.qp.assign(nql, {0, 0});
        for (int i = 0; i < nql; ++i)
            for (int h = 0; h < 2; ++h) {
                const std::pair<int, int> k{lv.quad[4 * i + 2 * h], lv.quad[4 * i + 2 * h + 1]};
                auto it = pid.find(k);
                if (it == pid.end()) {
                    it = pid.emplace(k, (int)dl.pairs.size()).first;
                    dl.pairs.push_back(k);
                }
                dl.qp[i][h] = it->second;
            }
        FBS_CUDA(cudaStreamSynchronize(lv.stream));  // the host tables go out of scope
    }
    ds->cnt.resize(ds->cnt128.size());
    for (size_t i = 0; i < ds->cnt.size(); ++i) ds->cnt[i] = u128_to_double(ds->cnt128[i]);
    ds->d_cnt = upload(p, ds->cnt);
    ds->d_num = (double *)p.dalloc(std::max<size_t>(1, ds->cnt.size()) * sizeof(double));
    ds->d_TD = (double *)p.dalloc(std::max<size_t>(1, ds->cnt.size()) * sizeof(double));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
}

// Shell fields of every bin of a level on its whole grid, then per group of
// pairs the forward transforms of their products, then the Gram products.
static void run_diagonal(Plan &p, const float *field) {
    DiagState &ds = *reinterpret_cast<DiagState *>(p.diag);
    const int nd = ds.nd;
    forward_or_follow(p, field);
    FBS_CUDA(cudaMemsetAsync(ds.d_num, 0, std::max<size_t>(1, ds.cnt.size()) * sizeof(double), p.stream));
    for (size_t l = 0; l < p.levels.size(); ++l) {
        Plan &lv = *p.levels[l];
        DiagLevel &dl = ds.lv[l];
        const int np = (int)dl.pairs.size();
        if (np == 0) continue;
        const int M = lv.M, nb = lv.nbins;
        const long long M3 = (long long)M * M * M;
        AsyncBuf Ifull((size_t)nb * M3 * sizeof(float), p.stream, "diagonal shell fields");
        AsyncBuf Gfull((size_t)dl.G_full * sizeof(float2), p.stream, "diagonal shell fields");
        AsyncBuf sq((size_t)nb * M * zstage_row_groups(M) * sizeof(double), p.stream, "diagonal shell fields");
        float2 *G0 = lv.d_G;
        const int slab0 = lv.slab;
        lv.d_G = Gfull.as<float2>();
        lv.slab = M;
        try {
            launch_inverse_x(lv, false);
            launch_inverse_yz_slab_geom(lv, 0, M, Ifull.as<float>(), dl.d_geom_full, nb, nb, sq.as<double>());
        } catch (...) {
            lv.d_G = G0;
            lv.slab = slab0;
            throw;
        }
        lv.d_G = G0;
        lv.slab = slab0;
        const long long per = (long long)dl.bx.D * dl.bx.D * dl.bx.Dz;  // complex elements of one pair spectrum
        const int K = (int)std::max<long long>(1, std::min<long long>(np, (4LL << 30) / (per * 8)));
        const int ng = (np + K - 1) / K;
        AsyncBuf prod((size_t)M3 * sizeof(float), p.stream, "diagonal scratch");
        AsyncBuf zb((size_t)M * M * dl.bx.Dz * sizeof(float2), p.stream, "diagonal scratch");
        AsyncBuf yb((size_t)M * dl.bx.D * dl.bx.Dz * sizeof(float2), p.stream, "diagonal scratch");
        AsyncBuf FA((size_t)std::min(np, K) * per * sizeof(float2), p.stream, "pair spectra");
        AsyncBuf FB(ng > 1 ? (size_t)K * per * sizeof(float2) : 16, p.stream, "pair spectra");
        const float *If = Ifull.as<float>();
        auto compute = [&](int g, float2 *dst) {
            for (int j = g * K; j < std::min(np, (g + 1) * K); ++j) {
                launch_field_product(lv, If + (long long)dl.pairs[j].first * M3, If + (long long)dl.pairs[j].second * M3,
                                     prod.as<float>(), M3);
                launch_forward_grid(lv, M, dl.bx, lv.fM, lv.d_twM, prod.as<float>(), nullptr, 1, zb.as<float2>(),
                                    yb.as<float2>(), dst + (long long)(j - g * K) * per);
            }
        };
        const double scale = 1.0 / ((double)M3 * (double)M3);  // DFT_M of a pair product is M^3 F_ab
        const int nql = (int)lv.nquad.size();
        for (int gi = 0; gi < ng; ++gi) {
            compute(gi, FA.as<float2>());
            for (int gj = gi; gj < ng; ++gj) {
                std::vector<long long> offs;
                std::vector<int> qout;
                for (int i = 0; i < nql; ++i) {
                    const int g0 = dl.qp[i][0] / K, g1 = dl.qp[i][1] / K;
                    int u, v;
                    if (g0 == gi && g1 == gj) {
                        u = dl.qp[i][0];
                        v = dl.qp[i][1];
                    } else if (g1 == gi && g0 == gj) {
                        u = dl.qp[i][1];
                        v = dl.qp[i][0];
                    } else {
                        continue;
                    }
                    offs.push_back((long long)(u - gi * K) * per);
                    offs.push_back((long long)(v - gj * K) * per);
                    qout.push_back(lv.gquad[i]);
                }
                if (qout.empty()) continue;
                const float2 *Bp = FA.as<float2>();
                if (gj != gi) {
                    compute(gj, FB.as<float2>());
                    Bp = FB.as<float2>();
                }
                for (size_t c0 = 0; c0 < qout.size(); c0 += 65535) {
                    const int nc = (int)std::min<size_t>(65535, qout.size() - c0);
                    AsyncBuf d_offs((size_t)nc * 2 * sizeof(long long), p.stream, "diagonal scratch");
                    AsyncBuf d_q((size_t)nc * sizeof(int), p.stream, "diagonal scratch");
                    FBS_CUDA(cudaMemcpyAsync(d_offs.ptr, offs.data() + 2 * c0, (size_t)nc * 2 * sizeof(long long),
                                             cudaMemcpyHostToDevice, p.stream));
                    FBS_CUDA(cudaMemcpyAsync(d_q.ptr, qout.data() + c0, (size_t)nc * sizeof(int),
                                             cudaMemcpyHostToDevice, p.stream));
                    launch_diag_gram(lv, FA.as<float2>(), Bp, d_offs.as<long long>(), nc, dl.d_idx, dl.d_w,
                                     dl.d_dstart, nd, d_q.as<int>(), scale, ds.d_num);
                    FBS_CUDA(cudaStreamSynchronize(p.stream));  // offs and qout go out of scope
                }
            }
        }
    }
    const double V = p.L * p.L * p.L, npix = (double)p.N * p.N * p.N;
    launch_diag_normalise(p, ds.d_num, ds.d_cnt, (long long)ds.cnt.size(), V * V * V / (npix * npix * npix * npix),
                          ds.d_TD);
}

// A tensor-core wait that gave up leaves a flag on the device; the outputs
// are NaN then (see the normalisation) and host-synchronising calls report it.
// Report (once) a timeout of any evaluation since the last report: waits for
// the plan's stream, reads the sticky flag and clears it.
static void check_device_errors(Plan &p) {
    int *f = tc_sticky_flag(p);
    if (!f) return;
    int v = 0;
    FBS_CUDA(cudaMemcpyAsync(&v, f, sizeof(int), cudaMemcpyDeviceToHost, p.stream));
    FBS_CUDA(cudaStreamSynchronize(p.stream));
    if (v) {
        FBS_CUDA(cudaMemsetAsync(f, 0, sizeof(int), p.stream));
        FBS_CUDA(cudaStreamSynchronize(p.stream));
        if (p.h_err) *p.h_err = 0;
        throw Failure{FBS_ERR_TIMEOUT, "a tensor-core pipeline wait of an evaluation on this plan timed out "
                                       "(code " + std::to_string(v) + "); its outputs are NaN"};
    }
}

// Without waiting: if an earlier evaluation is already known to have timed
// out (its status copy has landed in pinned host memory), report it now,
// before this call enqueues anything.  Skipped while the stream is being
// captured into a graph.
static void poll_device_errors(Plan &p) {
    if (!p.err_recorded || !p.h_err) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(p.stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cs != cudaStreamCaptureStatusNone) return;
    const cudaError_t q = cudaEventQuery(p.ev_err);
    if (q != cudaSuccess) {
        cudaGetLastError();  // cudaErrorNotReady: not known yet
        return;
    }
    if (*(volatile int *)p.h_err) check_device_errors(p);
}

// Pageable host memory (not registered with CUDA): the copy cannot run
// asynchronously, so the call waits for its results.
static bool is_pageable(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered;
}

static void copy_out(Plan &p, double *dst, const double *src, size_t n, bool &host) {
    if (!dst || n == 0) return;
    if (!is_device_ptr(dst) && is_pageable(dst)) host = true;
    FBS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, p.stream));
}

}  // namespace fbs

using namespace fbs;

struct fbs_plan : public fbs::Plan {};

#define FBS_GUARD_BEGIN try {
#define FBS_GUARD_END                                  \
    }                                                  \
    catch (const Failure &f) {                         \
        set_error(f.msg);                              \
        return f.status;                               \
    }                                                  \
    catch (const std::exception &e) {                  \
        set_error(std::string("internal: ") + e.what()); \
        return FBS_ERR_ARG;                            \
    }

extern "C" {

int fbs_version(void) { return 100; }

const char *fbs_last_error(void) { return g_last_error.c_str(); }

static const char *kClassNames[KC_NUM] = {"fwd_z",         "fwd_y",          "fwd_x",  "inv_x",
                                          "inv_y",         "inv_z",          "contract_fp32",
                                          "contract_tc",   "contract_quad",  "contract_quad_tc",
                                          "reduce",        "count"};

int fbs_num_kernel_classes(void) { return KC_NUM; }

const char *fbs_kernel_class_name(int i) { return (i >= 0 && i < KC_NUM) ? kClassNames[i] : ""; }

static fbs_status plan_create_impl(fbs_plan **out, int N, double L, const double *edges, int nbins,
                                   int precision, unsigned flags, void *cuda_stream, const void *blob,
                                   int64_t blob_size);

fbs_status fbs_plan_create(fbs_plan **out, int N, double L, const double *edges, int nbins,
                           int precision, unsigned flags, void *cuda_stream) {
    return plan_create_impl(out, N, L, edges, nbins, precision, flags, cuda_stream, nullptr, 0);
}

fbs_status fbs_plan_create_from_counts(fbs_plan **out, int N, double L, const double *edges, int nbins,
                                       int precision, unsigned flags, void *cuda_stream, const void *counts,
                                       int64_t size) {
    if (!counts || size <= 0) {
        if (out) *out = nullptr;
        set_error("counts blob is NULL or empty");
        return FBS_ERR_ARG;
    }
    return plan_create_impl(out, N, L, edges, nbins, precision, flags, cuda_stream, counts, size);
}

fbs_status fbs_plan_export_counts(const fbs_plan *plan, void *buf, int64_t *size) {
    if (!plan || !size) return FBS_ERR_ARG;
    const std::vector<unsigned char> b = export_counts(*plan);
    if (buf) {
        if (*size < (int64_t)b.size()) {
            set_error("buffer too small for the plan counts");
            *size = (int64_t)b.size();
            return FBS_ERR_ARG;
        }
        memcpy(buf, b.data(), b.size());
    }
    *size = (int64_t)b.size();
    return FBS_OK;
}

static fbs_status plan_create_impl(fbs_plan **out, int N, double L, const double *edges, int nbins,
                                   int precision, unsigned flags, void *cuda_stream, const void *blob,
                                   int64_t blob_size) {
    if (!out) {
        set_error("out is NULL");
        return FBS_ERR_ARG;
    }
    *out = nullptr;
    if (!edges || nbins < 1 || nbins > 128 || !(L > 0.0) || !isfinite(L)) {
        set_error("bad edges/nbins/L");
        return FBS_ERR_ARG;
    }
    if (precision < FBS_PREC_FP32 || precision > FBS_PREC_BF16) {
        set_error("unknown precision");
        return FBS_ERR_ARG;
    }
    for (int i = 0; i <= nbins; ++i)
        if (!isfinite(edges[i]) || edges[i] < 0.0 || (i > 0 && edges[i] < edges[i - 1])) {
            set_error("edges must be finite, non-negative and ascending");
            return FBS_ERR_ARG;
        }
    if (!good_N(N)) {
        set_error("N must be even, of the form 2^a 3^b, and in [8, 512]");
        return FBS_ERR_UNSUPPORTED_N;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return FBS_ERR_CUDA;
    }
    auto t0 = std::chrono::steady_clock::now();
    fbs_plan *p = new fbs_plan();
    p->N = N;
    p->L = L;
    p->nbins = nbins;
    p->precision = precision;
    p->flags = flags;
    p->stream = (cudaStream_t)cuda_stream;
    try {
        create_plan(*p, edges, blob, blob_size);
    } catch (const Failure &f) {
        set_error(f.msg);
        fbs_plan_free(p);
        return f.status;
    } catch (const std::exception &e) {
        set_error(std::string("internal: ") + e.what());
        fbs_plan_free(p);
        return FBS_ERR_ARG;
    }
    p->kt_ms[KC_COUNT] = 0;
    p->kt_n[KC_COUNT] = 0;
    p->pending.clear();
    p->create_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return FBS_OK;
}

void fbs_plan_free(fbs_plan *plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    if (plan->copy_stream) cudaStreamSynchronize(plan->copy_stream);
    cudaGetLastError();
    free_tc_state(*plan);
    free_batch(*plan);
    free_diag(*plan);
    for (Plan *lv : plan->levels) {
        free_tc_state(*lv);
        delete lv;
    }
    plan->levels.clear();
    for (void *ptr : plan->allocs) cudaFree(ptr);
    budget_release(plan->dev_bytes);
    if (plan->h_err) cudaFreeHost(plan->h_err);
    if (plan->ev_err) cudaEventDestroy(plan->ev_err);
    for (cudaEvent_t e : plan->evs) cudaEventDestroy(e);
    if (plan->ev_field_ready) cudaEventDestroy(plan->ev_field_ready);
    if (plan->ev_field_free) cudaEventDestroy(plan->ev_field_free);
    if (plan->copy_stream) cudaStreamDestroy(plan->copy_stream);
    cudaGetLastError();
    delete plan;
}

int fbs_plan_num_triplets(const fbs_plan *plan) {
    if (!plan) return FBS_ERR_ARG;
    return (int)plan->ntri.size();
}

int fbs_plan_num_quads(const fbs_plan *plan) {
    if (!plan) return FBS_ERR_ARG;
    return (int)plan->nquad.size();
}

fbs_status fbs_plan_triplets(const fbs_plan *plan, int32_t *abc, int64_t *ntri) {
    if (!plan) return FBS_ERR_ARG;
    if (abc && !plan->trip.empty()) memcpy(abc, plan->trip.data(), plan->trip.size() * sizeof(int32_t));
    if (ntri && !plan->ntri.empty()) memcpy(ntri, plan->ntri.data(), plan->ntri.size() * sizeof(int64_t));
    return FBS_OK;
}

fbs_status fbs_plan_quads(const fbs_plan *plan, int32_t *abcd, double *nq) {
    if (!plan) return FBS_ERR_ARG;
    if (abcd && !plan->quad.empty()) memcpy(abcd, plan->quad.data(), plan->quad.size() * sizeof(int32_t));
    if (nq && !plan->nquad.empty()) memcpy(nq, plan->nquad.data(), plan->nquad.size() * sizeof(double));
    return FBS_OK;
}

fbs_status fbs_plan_shells(const fbs_plan *plan, int64_t *sizes, int64_t *thr) {
    if (!plan) return FBS_ERR_ARG;
    for (int b = 0; b < plan->nbins && sizes; ++b) sizes[b] = plan->shell[b];
    for (int b = 0; b <= plan->nbins && thr; ++b) thr[b] = plan->thr[b];
    return FBS_OK;
}

fbs_status fbs_plan_set_precision(fbs_plan *plan, int precision) {
    if (!plan || precision < FBS_PREC_FP32 || precision > FBS_PREC_BF16) {
        set_error("bad plan or precision");
        return FBS_ERR_ARG;
    }
    plan->precision = precision;
    for (Plan *lv : plan->levels) lv->precision = precision;
    return FBS_OK;
}

static bool set_plan_option(Plan *plan, int option, int value);

fbs_status fbs_plan_set_option(fbs_plan *plan, int option, int value) {
    if (!plan) return FBS_ERR_ARG;
    if (!set_plan_option(plan, option, value)) {
        set_error("unknown option or value");
        return FBS_ERR_ARG;
    }
    FBS_GUARD_BEGIN
    if (option == FBS_OPT_SLAB_PLANES) FBS_CUDA(cudaStreamSynchronize(plan->stream));  // in-flight work uses the old layout
    for (Plan *lv : plan->levels) set_plan_option(lv, option, value);
    if (option == FBS_OPT_SLAB_PLANES && !plan->levels.empty()) {
        plan->slab = plan->levels.back()->slab;
        plan->nslabs = plan->levels.back()->nslabs;
    }
    return FBS_OK;
    FBS_GUARD_END
}

static bool set_plan_option(Plan *plan, int option, int value) {
    if (option == FBS_OPT_TC_WIDE && (value == 0 || value == 1)) {
        plan->tc_wide = value;
        return true;
    }
    if (option == FBS_OPT_TC_ROLES && value >= 0 && value <= 2) {
        plan->tc_roles = value;
        return true;
    }
    if (option == FBS_OPT_TC_CHUNK && value >= 0 && value <= 2) {
        plan->tc_chunk = value;
        return true;
    }
    if (option == FBS_OPT_TC_MERGE && (value == 0 || value == 1)) {
        plan->tc_merge = value;
        return true;
    }
    if (option == FBS_OPT_TC_BSTAGES && (value == 0 || (value >= 2 && value <= 4))) {
        plan->tc_bstages = value;
        return true;
    }
    if (option == FBS_OPT_TC_BFROMA && (value == 0 || value == 1)) {
        plan->tc_bfroma = value;
        return true;
    }
    if (option == FBS_OPT_TC_STACK && (value == 0 || value == 1)) {
        plan->tc_stack = value;
        return true;
    }
    if (option == FBS_OPT_TC_PAIRS && (value == 0 || value == 1)) {
        plan->tc_pairs = value;
        return true;
    }
    if (option == FBS_OPT_TC_WAIT_LIMIT && value >= 0) {
        plan->tc_wait_limit = value;
        return true;
    }
    if (option == FBS_OPT_SLAB_PLANES && value >= 0) {
        if (plan->root_) {  // a level: fewer planes per slab in the same buffers
            plan->slab = value > 0 ? std::min(value, plan->slab_planned) : plan->slab_planned;
            plan->nslabs = (plan->M + plan->slab - 1) / plan->slab;
            set_slab_offsets(*plan);
        }
        return true;
    }
    return false;
}

fbs_status fbs_plan_set_stream(fbs_plan *plan, void *stream) {
    if (!plan) return FBS_ERR_ARG;
    FBS_GUARD_BEGIN
    plan->flush_times();
    FBS_CUDA(cudaStreamSynchronize(plan->stream));
    plan->stream = (cudaStream_t)stream;
    for (Plan *lv : plan->levels) lv->stream = plan->stream;
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_plan_tc_info(const fbs_plan *plan, int level, int which, int32_t *info) {
    if (!plan || !info || level < 0 || level >= (int)plan->levels.size() || which < 0 || which > 2) {
        set_error("fbs_plan_tc_info: bad argument");
        return FBS_ERR_ARG;
    }
    tc_job_info(*plan->levels[level], which, info);
    return FBS_OK;
}

fbs_status fbs_plan_follow(fbs_plan *follower, const fbs_plan *leader) {
    if (!follower || follower == leader) {
        set_error("fbs_plan_follow: bad plan");
        return FBS_ERR_ARG;
    }
    FBS_GUARD_BEGIN
    FBS_CUDA(cudaStreamSynchronize(follower->stream));
    Plan &f = *follower;
    if (!f.own_box) {
        f.own_box = f.d_box;
        f.own_boxgeom = f.box;
    }
    if (!leader) {  // detach: the plan's own box again
        f.leader = nullptr;
        f.d_box = f.own_box;
        f.box = f.own_boxgeom;
    } else {
        if (leader->leader) throw Failure{FBS_ERR_ARG, "fbs_plan_follow: the leader follows another plan"};
        if (leader->N != f.N) throw Failure{FBS_ERR_ARG, "fbs_plan_follow: grids differ"};
        if (leader->box.R < f.own_boxgeom.R)
            throw Failure{FBS_ERR_ARG, "fbs_plan_follow: the leader's spectrum box is smaller than the follower's"};
        if (leader->stream != f.stream) throw Failure{FBS_ERR_STATE, "fbs_plan_follow: the plans' streams differ"};
        f.leader = leader;
        f.d_box = leader->d_box;
        f.box = leader->box;
    }
    for (Plan *lv : f.levels) {
        lv->d_box = f.d_box;
        lv->box = f.box;
        lv->boxM = f.box;
        lv->boxM.N = lv->M;
    }
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_bispectrum(fbs_plan *plan, const float *field, double *B, double *P) {
    if (!plan || (!field && !plan->leader)) {
        set_error("plan or field is NULL");
        return FBS_ERR_ARG;
    }
    FBS_GUARD_BEGIN
    poll_device_errors(*plan);
    run_field(*plan, field, false);
    bool host = false;
    copy_out(*plan, B, plan->d_B, plan->ntri.size(), host);
    copy_out(*plan, P, plan->d_P, plan->nbins, host);
    if (host) {
        FBS_CUDA(cudaStreamSynchronize(plan->stream));
        check_device_errors(*plan);
    }
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_trispectrum(fbs_plan *plan, const float *field, double *T, double *B, double *P) {
    if (!plan || (!field && !plan->leader)) {
        set_error("plan or field is NULL");
        return FBS_ERR_ARG;
    }
    if (!(plan->flags & FBS_FLAG_TRISPECTRUM)) {
        set_error("plan was created without FBS_FLAG_TRISPECTRUM");
        return FBS_ERR_STATE;
    }
    FBS_GUARD_BEGIN
    poll_device_errors(*plan);
    run_field(*plan, field, true);
    bool host = false;
    copy_out(*plan, T, plan->d_T, plan->nquad.size(), host);
    copy_out(*plan, B, plan->d_B, plan->ntri.size(), host);
    copy_out(*plan, P, plan->d_P, plan->nbins, host);
    if (host) {
        FBS_CUDA(cudaStreamSynchronize(plan->stream));
        check_device_errors(*plan);
    }
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_bispectrum_batch(fbs_plan *plan, const float *const *fields, int nfields, double *B, double *P) {
    if (!plan || !fields || nfields < 1 || nfields > 65535 / std::max(1, plan->nbins)) {
        set_error("bad plan, field list or batch size");
        return FBS_ERR_ARG;
    }
    for (int f = 0; f < nfields; ++f)
        if (!fields[f] || !is_device_ptr(fields[f])) {
            set_error("batched fields must be device pointers");
            return FBS_ERR_ARG;
        }
    FBS_GUARD_BEGIN
    poll_device_errors(*plan);
    run_batch(*plan, fields, nfields);
    BatchState &bs = *reinterpret_cast<BatchState *>(plan->batch);
    bool host = false;
    copy_out(*plan, B, bs.B, (size_t)nfields * plan->ntri.size(), host);
    copy_out(*plan, P, bs.P, (size_t)nfields * plan->nbins, host);
    if (host) {
        FBS_CUDA(cudaStreamSynchronize(plan->stream));
        check_device_errors(*plan);
    }
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_plan_set_diagonal(fbs_plan *plan, const double *diag_edges, int ndiag) {
    if (!plan || !diag_edges || ndiag < 1 || ndiag > 4096) {
        set_error("fbs_plan_set_diagonal: bad argument");
        return FBS_ERR_ARG;
    }
    if (!(plan->flags & FBS_FLAG_TRISPECTRUM)) {
        set_error("plan was created without FBS_FLAG_TRISPECTRUM");
        return FBS_ERR_STATE;
    }
    FBS_GUARD_BEGIN
    FBS_CUDA(cudaStreamSynchronize(plan->stream));
    set_diagonal(*plan, diag_edges, ndiag);
    return FBS_OK;
    FBS_GUARD_END
}

int fbs_plan_num_diagonal_bins(const fbs_plan *plan) {
    if (!plan) return FBS_ERR_ARG;
    return plan->diag ? reinterpret_cast<const DiagState *>(plan->diag)->nd : 0;
}

fbs_status fbs_plan_diagonal_counts(const fbs_plan *plan, double *counts, uint64_t *words) {
    if (!plan || !plan->diag) {
        set_error("fbs_plan_diagonal_counts: no diagonal bins set");
        return plan ? FBS_ERR_STATE : FBS_ERR_ARG;
    }
    const DiagState &ds = *reinterpret_cast<const DiagState *>(plan->diag);
    for (size_t i = 0; i < ds.cnt128.size(); ++i) {
        if (counts) counts[i] = ds.cnt[i];
        if (words) {
            words[2 * i] = ds.cnt128[i].lo;
            words[2 * i + 1] = ds.cnt128[i].hi;
        }
    }
    return FBS_OK;
}

fbs_status fbs_trispectrum_diagonal(fbs_plan *plan, const float *field, double *TD) {
    if (!plan || (!field && !plan->leader) || !TD) {
        set_error("fbs_trispectrum_diagonal: NULL argument");
        return FBS_ERR_ARG;
    }
    if (!plan->diag) {
        set_error("fbs_trispectrum_diagonal: call fbs_plan_set_diagonal first");
        return FBS_ERR_STATE;
    }
    FBS_GUARD_BEGIN
    poll_device_errors(*plan);
    run_diagonal(*plan, field);
    const DiagState &ds = *reinterpret_cast<const DiagState *>(plan->diag);
    bool host = false;
    copy_out(*plan, TD, ds.d_TD, ds.cnt.size(), host);
    if (host) FBS_CUDA(cudaStreamSynchronize(plan->stream));
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_trispectrum_connected(fbs_plan *plan, const float *field, double *Tc, double *T, double *B,
                                     double *P) {
    if (!plan || (!field && !plan->leader)) {
        set_error("plan or field is NULL");
        return FBS_ERR_ARG;
    }
    if (!(plan->flags & FBS_FLAG_TRISPECTRUM)) {
        set_error("plan was created without FBS_FLAG_TRISPECTRUM");
        return FBS_ERR_STATE;
    }
    FBS_GUARD_BEGIN
    poll_device_errors(*plan);
    run_field(*plan, field, true);
    if (!plan->nquad.empty()) launch_connected(*plan, plan->d_Tc);
    bool host = false;
    copy_out(*plan, Tc, plan->d_Tc, plan->nquad.size(), host);
    copy_out(*plan, T, plan->d_T, plan->nquad.size(), host);
    copy_out(*plan, B, plan->d_B, plan->ntri.size(), host);
    copy_out(*plan, P, plan->d_P, plan->nbins, host);
    if (host) {
        FBS_CUDA(cudaStreamSynchronize(plan->stream));
        check_device_errors(*plan);
    }
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_plan_triangle_average(fbs_plan *plan, const double *w, int nfunc, int64_t nw, const int32_t *terms,
                                     const double *coef, int nterms, double *out) {
    if (!plan || !w || nfunc < 1 || !terms || !coef || nterms < 1 || !out) {
        set_error("fbs_plan_triangle_average: bad argument");
        return FBS_ERR_ARG;
    }
    if (nw < plan->thr[plan->nbins]) {
        set_error("weight tables must cover every |m|^2 below the top edge (nw >= " +
                  std::to_string(plan->thr[plan->nbins]) + ")");
        return FBS_ERR_ARG;
    }
    for (int k = 0; k < 3 * nterms; ++k)
        if (terms[k] < 0 || terms[k] >= nfunc) {
            set_error("fbs_plan_triangle_average: term names a function outside [0, nfunc)");
            return FBS_ERR_ARG;
        }
    FBS_GUARD_BEGIN
    FBS_CUDA(cudaStreamSynchronize(plan->stream));
    // the tables, on the device for the weighted count fields
    AsyncBuf wbuf((size_t)nfunc * nw * sizeof(double), plan->stream, "weight tables");
    FBS_CUDA(cudaMemcpyAsync(wbuf.ptr, w, (size_t)nfunc * nw * sizeof(double), cudaMemcpyHostToDevice, plan->stream));
    std::vector<double> acc(plan->ntri.size(), 0.0);
    for (Plan *lp : plan->levels) {
        Plan &lv = *lp;
        const int nt = (int)lv.ntri.size();
        if (nt == 0) continue;
        // only the functions some term uses get fields
        std::vector<int> fmap(nfunc, -1);
        std::vector<const double *> tabs;
        for (int k = 0; k < 3 * nterms; ++k)
            if (fmap[terms[k]] < 0) {
                fmap[terms[k]] = (int)tabs.size();
                tabs.push_back(wbuf.as<double>() + (size_t)terms[k] * nw);
            }
        std::vector<int> items;
        items.reserve((size_t)nt * nterms * 3);
        for (int t = 0; t < nt; ++t)
            for (int k = 0; k < nterms; ++k)
                for (int j = 0; j < 3; ++j) items.push_back(fmap[terms[3 * k + j]] * lv.nbins + lv.trip[3 * t + j]);
        std::vector<double> sums;
        octant_sums(lv, tabs, items, 3, sums);
        // sum over the M^3 grid / M^3 = the sum over the closed ordered triples
        const double npix = (double)lv.M * lv.M * lv.M;
        for (int t = 0; t < nt; ++t) {
            double v = 0.0;
            for (int k = 0; k < nterms; ++k) v += coef[k] * sums[(size_t)t * nterms + k];
            acc[lv.gtrip[t]] = v / npix / (double)lv.ntri[t];
        }
    }
    memcpy(out, acc.data(), acc.size() * sizeof(double));
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_plan_shell_average(const fbs_plan *plan, const double *w, int64_t nw, double *out) {
    if (!plan || !w || !out) return FBS_ERR_ARG;
    const int N = plan->N, nb = plan->nbins;
    const long long top = plan->thr[nb];
    if (nw < top) {
        set_error("the table must cover every |m|^2 below the top edge");
        return FBS_ERR_ARG;
    }
    // every lattice mode with components in [-N/2, N/2), by bin
    std::vector<double> sum(nb, 0.0);
    std::vector<long long> cnt(nb, 0);
    std::vector<int> lut((size_t)std::max<long long>(top, 1), -1);
    for (int b = 0; b < nb; ++b)
        for (long long v = plan->thr[b]; v < plan->thr[b + 1]; ++v) lut[v] = b;
    const int Rm = std::min(isqrt_floor(top - 1), N / 2);
    for (int x = -Rm; x <= std::min(Rm, N / 2 - 1); ++x)
        for (int y = -Rm; y <= std::min(Rm, N / 2 - 1); ++y)
            for (int z = -Rm; z <= std::min(Rm, N / 2 - 1); ++z) {
                const long long v = (long long)x * x + (long long)y * y + (long long)z * z;
                if (v >= top || lut[v] < 0) continue;
                sum[lut[v]] += w[v];
                cnt[lut[v]] += 1;
            }
    for (int b = 0; b < nb; ++b) out[b] = cnt[b] ? sum[b] / (double)cnt[b] : nan("");
    return FBS_OK;
}

fbs_status fbs_plan_quads_connected(const fbs_plan *plan, double *nconn) {
    if (!plan) return FBS_ERR_ARG;
    if (nconn && !plan->nconn.empty()) memcpy(nconn, plan->nconn.data(), plan->nconn.size() * sizeof(double));
    return FBS_OK;
}

fbs_status fbs_plan_sums(fbs_plan *plan, double *num_trip, double *num_quad, double *sumsq) {
    if (!plan) return FBS_ERR_ARG;
    FBS_GUARD_BEGIN
    if (num_trip && !plan->ntri.empty())
        FBS_CUDA(cudaMemcpyAsync(num_trip, plan->d_tnum, plan->ntri.size() * sizeof(double),
                                 cudaMemcpyDefault, plan->stream));
    if (num_quad && !plan->nquad.empty())
        FBS_CUDA(cudaMemcpyAsync(num_quad, plan->d_qnum, plan->nquad.size() * sizeof(double),
                                 cudaMemcpyDefault, plan->stream));
    if (sumsq)
        FBS_CUDA(cudaMemcpyAsync(sumsq, plan->d_sumsq, plan->nbins * sizeof(double), cudaMemcpyDefault,
                                 plan->stream));
    FBS_CUDA(cudaStreamSynchronize(plan->stream));
    check_device_errors(*plan);
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_plan_check(fbs_plan *plan) {
    if (!plan) return FBS_ERR_ARG;
    FBS_GUARD_BEGIN
    FBS_CUDA(cudaStreamSynchronize(plan->stream));
    check_device_errors(*plan);
    return FBS_OK;
    FBS_GUARD_END
}

fbs_status fbs_set_device_budget(int64_t bytes) {
    if (bytes < 0) {
        set_error("budget must be >= 0");
        return FBS_ERR_ARG;
    }
    g_budget.store(bytes);
    return FBS_OK;
}

int64_t fbs_device_bytes_in_use(void) { return g_in_use.load(); }

fbs_status fbs_set_slab_budget(int64_t bytes) {
    if (bytes < 0) {
        set_error("slab budget must be >= 0");
        return FBS_ERR_ARG;
    }
    g_slab_default.store(bytes);
    return FBS_OK;
}

fbs_status fbs_plan_kernel_times(fbs_plan *plan, double *ms, int64_t *launches, int reset) {
    if (!plan) return FBS_ERR_ARG;
    FBS_GUARD_BEGIN
    plan->flush_times();
    for (int i = 0; i < KC_NUM; ++i) {
        if (ms) ms[i] = plan->kt_ms[i];
        if (launches) launches[i] = plan->kt_n[i];
        if (reset) {
            plan->kt_ms[i] = 0;
            plan->kt_n[i] = 0;
        }
    }
    return FBS_OK;
    FBS_GUARD_END
}

double fbs_plan_create_ms(const fbs_plan *plan) { return plan ? plan->create_ms : -1.0; }

double fbs_plan_count_margin(const fbs_plan *plan) { return plan ? plan->count_margin : -1.0; }

int fbs_plan_eval_grid(const fbs_plan *plan) { return plan ? plan->M : FBS_ERR_ARG; }

fbs_status fbs_plan_item_levels(const fbs_plan *plan, int32_t *trip_level, int32_t *quad_level) {
    if (!plan) return FBS_ERR_ARG;
    for (size_t l = 0; l < plan->levels.size(); ++l) {
        const Plan &lv = *plan->levels[l];
        if (trip_level)
            for (int g : lv.gtrip) trip_level[g] = (int32_t)l;
        if (quad_level)
            for (int g : lv.gquad) quad_level[g] = (int32_t)l;
    }
    return FBS_OK;
}

int fbs_plan_num_levels(const fbs_plan *plan) { return plan ? (int)plan->levels.size() : FBS_ERR_ARG; }

fbs_status fbs_plan_level(const fbs_plan *plan, int i, int *M, int *nbins, int *ntrip, int *nquad,
                          int *slab_planes, int *nslabs) {
    if (!plan || i < 0 || i >= (int)plan->levels.size()) {
        set_error("bad plan or level index");
        return FBS_ERR_ARG;
    }
    const Plan &lv = *plan->levels[i];
    if (M) *M = lv.M;
    if (nbins) *nbins = lv.nbins;
    if (ntrip) *ntrip = (int)lv.ntri.size();
    if (nquad) *nquad = (int)lv.nquad.size();
    if (slab_planes) *slab_planes = lv.slab;
    if (nslabs) *nslabs = lv.nslabs;
    return FBS_OK;
}

int fbs_plan_slab_planes(const fbs_plan *plan) { return plan ? plan->slab : FBS_ERR_ARG; }

int fbs_plan_num_slabs(const fbs_plan *plan) { return plan ? plan->nslabs : FBS_ERR_ARG; }

int fbs_plan_quad_counts_exact(const fbs_plan *plan) { return plan ? 1 : FBS_ERR_ARG; }

fbs_status fbs_plan_quad_counts_u128(const fbs_plan *plan, uint64_t *words) {
    if (!plan || !words) {
        set_error("fbs_plan_quad_counts_u128: NULL argument");
        return FBS_ERR_ARG;
    }
    for (size_t i = 0; i < plan->nquad128.size(); ++i) {
        words[2 * i] = plan->nquad128[i].lo;
        words[2 * i + 1] = plan->nquad128[i].hi;
    }
    return FBS_OK;
}

int64_t fbs_plan_device_bytes(const fbs_plan *plan) { return plan ? plan->dev_bytes : -1; }

}  // extern "C"
