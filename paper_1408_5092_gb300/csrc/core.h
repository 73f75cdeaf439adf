// Core types of the MPS-PT library: quantum numbers, bond bases, errors,
// stream-ordered device buffers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <shared_mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mpspt.h"

namespace mpspt {

struct Error : std::runtime_error {
    mpspt_status status;
    Error(mpspt_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define MPSPT_CUDA(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (e_ == cudaErrorMemoryAllocation)                                          \
                throw ::mpspt::Error(MPSPT_ERR_OOM, std::string(#call) + ": " +           \
                                                        cudaGetErrorString(e_));          \
            throw ::mpspt::Error(MPSPT_ERR_CUDA,                                          \
                                 std::string(#call) + ": " + cudaGetErrorString(e_));     \
        }                                                                                 \
    } while (0)

inline void require(bool ok, const std::string& msg, mpspt_status s = MPSPT_ERR_INVALID) {
    if (!ok) throw Error(s, msg);
}

// (N, 2Sz) of a left part of the chain, or a change of it.
struct QN {
    int n = 0, sz = 0;
    QN() = default;
    QN(int n_, int sz_) : n(n_), sz(sz_) {}
    QN operator+(const QN& o) const { return {n + o.n, sz + o.sz}; }
    QN operator-(const QN& o) const { return {n - o.n, sz - o.sz}; }
    bool operator==(const QN& o) const { return n == o.n && sz == o.sz; }
    bool operator!=(const QN& o) const { return !(*this == o); }
    bool operator<(const QN& o) const { return n < o.n || (n == o.n && sz < o.sz); }
};

// Local site basis |0>, |a>, |b>, |ab>.
inline QN site_qn(int s) {
    static const int N[4] = {0, 1, 1, 2};
    static const int S[4] = {0, 1, -1, 0};
    return {N[s], S[s]};
}

struct Sector {
    QN q;
    int dim = 0;
    int off = 0;  // position of the sector's first index in the bond basis
};

// Bond basis at one cut: QN sectors sorted ascending, contiguous indices.
struct Bond {
    std::vector<Sector> sec;
    int total = 0;
    int find(const QN& q) const {
        int lo = 0, hi = (int)sec.size() - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            if (sec[mid].q == q) return mid;
            if (sec[mid].q < q) lo = mid + 1; else hi = mid - 1;
        }
        return -1;
    }
    void finalize() {
        total = 0;
        for (auto& s : sec) { s.off = total; total += s.dim; }
    }
    int nsec() const { return (int)sec.size(); }
};

// Registry of live device allocations.  Task lists are validated against it
// before launch (every pointer range a kernel will touch must lie inside one
// live allocation), so a planner error becomes a status, not a bad access.
struct Registry {
    // Readers (the planners' range checks, many per task list and from every
    // lane thread) share the lock; allocations and releases take it alone.
    // Each thread remembers the last few allocations it found; the memory
    // is valid until any allocation is released (gen counts releases).
    std::shared_mutex mu;
    std::map<uintptr_t, size_t> live;
    std::atomic<unsigned long long> gen{0};
    static Registry& get() { static Registry r; return r; }
    void add(const void* p, size_t n) { std::unique_lock<std::shared_mutex> g(mu); live[(uintptr_t)p] = n; }
    void remove(const void* p) {
        std::unique_lock<std::shared_mutex> g(mu);
        live.erase((uintptr_t)p);
        gen.fetch_add(1, std::memory_order_release);
    }
    bool contains(const void* p, size_t bytes) {
        constexpr int kWays = 8;
        thread_local uintptr_t c0[kWays] = {}, c1[kWays] = {};
        thread_local unsigned long long cg = ~0ULL;
        thread_local int next = 0;
        const uintptr_t a = (uintptr_t)p, b = a + bytes;
        const unsigned long long g0 = gen.load(std::memory_order_acquire);
        if (cg == g0)
            for (int w = 0; w < kWays; ++w)
                if (a >= c0[w] && b <= c1[w]) return true;
        std::shared_lock<std::shared_mutex> g(mu);
        auto it = live.upper_bound(a);
        if (it == live.begin()) return false;
        --it;
        if (!(a >= it->first && b <= it->first + it->second)) return false;
        if (cg != g0) {   // a release happened: forget everything remembered
            for (int w = 0; w < kWays; ++w) c0[w] = c1[w] = 0;
            cg = g0;
        }
        c0[next] = it->first;
        c1[next] = it->first + it->second;
        next = (next + 1) % kWays;
        return true;
    }
};

// Bounds checks are on unless MPSPT_CHECK=0.
inline bool checks_enabled() {
    static int on = [] { const char* e = std::getenv("MPSPT_CHECK"); return (e && e[0] == '0') ? 0 : 1; }();
    return on != 0;
}

inline void check_range(const void* p, size_t bytes, const char* what) {
    if (!checks_enabled() || bytes == 0) return;
    if (!Registry::get().contains(p, bytes))
        throw Error(MPSPT_ERR_INVALID, std::string("planner bounds check failed: ") + what);
}

// The library allocates from the device's default memory pool.  Its release
// threshold is raised so that freed blocks stay cached in the pool across
// stream synchronisations (by default they return to the driver at every
// sync and the next allocations remap them, which dominated planning time).
// This is a property of this process's pool, not a device setting.
inline void keep_pool_memory(int device) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return;
    unsigned long long thr = ~0ULL;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

// Stream-ordered device allocation (cudaMallocAsync), released on the same
// stream.  Sizes in bytes.
class DBuf {
  public:
    DBuf() = default;
    DBuf(size_t bytes, cudaStream_t st) { alloc(bytes, st); }
    ~DBuf() { release(); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = std::move(o); }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p_ = o.p_; n_ = o.n_; st_ = o.st_; owned_ = o.owned_;
            o.p_ = nullptr; o.n_ = 0; o.owned_ = true;
        }
        return *this;
    }
    void alloc(size_t bytes, cudaStream_t st) {
        release();
        st_ = st;
        n_ = bytes;
        if (bytes) {
            MPSPT_CUDA(cudaMallocAsync(&p_, bytes, st));
            Registry::get().add(p_, bytes);
        }
    }
    void ensure(size_t bytes, cudaStream_t st) {
        if (bytes > n_) alloc(bytes + bytes / 4, st);
    }
    void release() {
        if (p_ && owned_) { Registry::get().remove(p_); cudaFreeAsync(p_, st_); }
        p_ = nullptr;
        n_ = 0;
        owned_ = true;
    }
    // non-owning view of memory owned by another buffer
    void make_view(void* p, size_t bytes) {
        release();
        p_ = p;
        n_ = bytes;
        owned_ = false;
    }
    template <class T> T* as() const { return static_cast<T*>(p_); }
    void* get() const { return p_; }
    size_t bytes() const { return n_; }

  private:
    void* p_ = nullptr;
    size_t n_ = 0;
    cudaStream_t st_ = 0;
    bool owned_ = true;
};

// Pinned staging ring of one stream.  A host-to-device copy from pageable
// memory goes through the driver's own staging buffer, which every host
// thread of the process shares; concurrent lanes then serialise on it, and
// the copy blocks the calling thread.  Task lists are instead copied into
// this ring (page-locked) and sent with a truly asynchronous copy.  The ring
// has two halves; before a half is written again, the event recorded when
// the previous half was left is waited on, so the copies from it are done.
struct PinnedRing {
    unsigned char* base = nullptr;
    size_t half = 0, off = 0;
    int cur = 0;
    bool used[2] = {false, false};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaStream_t st = 0;
    PinnedRing(size_t bytes, cudaStream_t s) : st(s) {
        half = bytes / 2;
        MPSPT_CUDA(cudaMallocHost(&base, 2 * half));
        MPSPT_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        MPSPT_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    }
    ~PinnedRing() {
        cudaStreamSynchronize(st);
        if (base) cudaFreeHost(base);
        for (auto& e : ev) if (e) cudaEventDestroy(e);
    }
    PinnedRing(const PinnedRing&) = delete;
    PinnedRing& operator=(const PinnedRing&) = delete;
    // page-locked copy of src (nullptr if it does not fit in a half)
    void* stage(const void* src, size_t n) {
        const size_t need = (n + 255) & ~(size_t)255;
        if (need > half) return nullptr;
        if (off + need > half) {
            MPSPT_CUDA(cudaEventRecord(ev[cur], st));
            used[cur] = true;
            cur ^= 1;
            if (used[cur]) MPSPT_CUDA(cudaEventSynchronize(ev[cur]));
            off = 0;
        }
        unsigned char* p = base + (size_t)cur * half + off;
        std::memcpy(p, src, n);
        off += need;
        return p;
    }
};

// The staging ring of the calling thread's current lane (set by the sweep
// drivers for their duration; null = plain pageable copies).
inline PinnedRing*& thread_ring() {
    thread_local PinnedRing* r = nullptr;
    return r;
}

struct RingScope {
    PinnedRing* prev;
    explicit RingScope(PinnedRing* r) : prev(thread_ring()) { thread_ring() = r; }
    ~RingScope() { thread_ring() = prev; }
};

inline void copy_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (!bytes) return;
    PinnedRing* r = thread_ring();
    if (r && r->st == st) {
        if (void* p = r->stage(src, bytes)) {
            MPSPT_CUDA(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, st));
            return;
        }
    }
    MPSPT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
}

template <class T>
inline void upload(DBuf& dst, const std::vector<T>& v, cudaStream_t st) {
    dst.ensure(v.size() * sizeof(T) + 16, st);
    if (!v.empty()) copy_h2d(dst.get(), v.data(), v.size() * sizeof(T), st);
}

}  // namespace mpspt
