// Forward y pass and z pass in one persistent kernel (transform path 2).
//
// The two-field intermediate of one k_x plane (W and Y^X^V_z, 2 x n_y x n_z
// complex) goes from the y tiles to the z tiles through a ring of R k_x
// planes (about 40 MB: R = 40 at 256^3) that stays in L2, instead of through
// HBM (85 MB written and read per 256^3 frame on the five-pass path).  The
// per-line arithmetic is that of k_fy and k_fz with 16 lines per tile (the
// same operations as the five-pass path with the tile plan (16, 16, *); the
// compiler may contract them differently, so the two agree to rounding).
//
// Work comes from a ticket in this order: iteration i holds the y tiles of
// k_x = i (one per live 16-plane z-slab) and then the z tiles of
// k_x = i - lag (one per 16 k_y), lag = R / 2.  A z tile of k_x waits until
// every y tile of k_x is done; a y tile of k_x >= R waits until every z tile
// of k_x - R is done (its ring plane is free).  The ring and the lag are as
// large as they are so that the window of tickets the resident CTAs hold
// (12 to 24 iterations at 256^3: 304 CTAs, each with its current ticket and
// the next) rarely waits at all.  Both wait only on tiles of earlier tickets,
// which running CTAs hold, so the waits end; each is bounded all the same
// (about 0.4 s, then the error flag and on).  A y tile's three component
// tiles come in by bulk copies issued before its wait; ring data written by
// other CTAs is read through L2 (ld.global.cg), never from L1.
#include "fft_common.cuh"
#include "ftr_internal.h"
#include "tc_sm100.cuh"

namespace ftr {
namespace {

constexpr int kF = 16;                      // lines per tile
constexpr size_t kRingBytes = 40u << 20;    // ring target: about 40 MB of the 129 MB L2
constexpr unsigned kSpinLimit = 1u << 22;   // polls of a dependency wait (~0.4 s)

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until *cnt >= need (bounded); then the whole CTA proceeds.
__device__ __forceinline__ void wait_count(const int* cnt, int need, int* err) {
    if (threadIdx.x == 0) {
        unsigned it = 0;
        while (ld_acquire(cnt) < need) {
            if (++it > kSpinLimit) {
                atomicExch(err, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
    }
    __syncthreads();
}

// Count the CTA's previous tile as done (its counter in *pend, if any).
// Called at the start of the next tile, after that tile's copies are issued,
// so that the fence's wait for the stores overlaps the fetch.  The barrier
// that ended the previous tile ordered every thread's stores before thread
// 0 (CTA scope); its fence makes them visible GPU-wide ahead of the count.
// The call precedes every wait of the new tile, so a tile never waits while
// its own CTA holds back a count.
__device__ __forceinline__ void raise_pending(int*& pend) {
    if (threadIdx.x == 0 && pend) {
        __threadfence();
        atomicAdd(pend, 1);
    }
    pend = nullptr;
}

// Wait for a bulk copy's completion; past the limit the error flag is set
// and the copy is waited for once more (bounded), so that none is left in
// flight into this CTA's shared memory.
__device__ __forceinline__ void wait_copy(uint64_t* mbar, uint32_t parity, int* err) {
    if (!tc::mbar_wait(mbar, parity, kSpinLimit)) {
        atomicExch(err, 1);
        tc::mbar_wait(mbar, parity, kSpinLimit);
    }
}

// Line f's elements z = N2 n1 + r of a staged 16-line tile B (zero outside
// the live range [zl, zh): the ring holds older planes' values there), then
// step 1 with B itself as the exchange buffer.
template <int N>
__device__ __forceinline__ void zstaged_step1(float2* B, int r, int f, int zl, int zh,
                                              const float2* __restrict__ tw) {
    using X = Xchg<N, kF>;
    float2 v[X::N1];
    if (r < X::N2) {
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int z = X::N2 * n1 + r;
            v[n1] = (z >= zl && z < zh) ? B[f * N + z] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();                             // the staged lines are in registers: B becomes the exchange
    if (r < X::N2) fft_step1<N, kF, -1>(v, f, r, B, tw);
}

// n_y = n_z = N.  sync: [0] ticket, [1 .. nkx] y tiles done per k_x,
// [1 + nkx .. 2 nkx] z tiles done per k_x (all zero at launch).
// CTAs per SM the register budget asks for: two for 128 <= N <= 256 (the
// shared memory of three 16-line component tiles allows two at N = 256, and
// three spill the y and z code paths held in one kernel), else that of the
// axis passes
template <int N>
struct YzMinCtas {
    static constexpr int value = (N >= 128 && N <= 256) ? 2 : MinCtasF<N, kF>::value;
};

// One of the three shared-memory buffers: a component's staged 16-line tile,
// then its exchange buffer (and the stash of the transformed x component).
template <int N>
struct YzBuf {
    static constexpr int value = cmax(Xchg<N, kF>::SIZE, (kF + 1) * N);
};

template <int N>
__global__ void __launch_bounds__(kF * Xchg<N, kF>::NT, YzMinCtas<N>::value)
    k_fyz(GridDev g, const float2* __restrict__ s0, float2* __restrict__ s1, float2* ring, int kRing, int kLag,
          int64_t Mh, const float2* __restrict__ twy, const float2* __restrict__ twz, float wx_scale, float wy_scale,
          float wz_scale, float inv_m, const int* __restrict__ meta, int* sync, int* err) {
    pdl_wait();
    using X = Xchg<N, kF>;
    constexpr int BUF = YzBuf<N>::value;
    constexpr uint32_t kBytes = kF * N * sizeof(float2);
    extern __shared__ __align__(16) float2 smem[];
    __shared__ uint64_t mbar[3];
    __shared__ int s_ticket[2];
    const int nz = N, ny = N;
    const int nkx = g.n[0] / 2 + 1;
    int zl, zh;
    live_z_range(meta, zl, zh);
    const int nslab = (zh - zl) / kF;            // y tiles per k_x
    const int nzt = ny / kF;                     // z tiles per k_x
    const int64_t total = (int64_t)nkx * (nslab + nzt);
    const size_t plane = (size_t)ny * nz;        // one field of one ring plane
    int* ydone = sync + 1;
    int* zdone = sync + 1 + nkx;
    const int tid = threadIdx.x;
    const uint64_t pout = l2_evict_last();
    if (tid == 0) {
        for (int c = 0; c < 3; ++c) tc::mbar_init(&mbar[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ticket[0] = atomicAdd(&sync[0], 1);
    }
    __syncthreads();
    int slot = 0;
    int64_t t = s_ticket[0];
    uint32_t par = 0;                            // bit c: parity of copy barrier c's next phase
    int* pend = nullptr;                         // done-counter of the previous tile, not yet raised
    for (;;) {
        if (t >= total) break;
        // the next ticket is taken now and kept in thread 0's register, so
        // its round trip overlaps this tile (a CTA holding a ticket it has
        // not started has a current one below it, so the smallest open
        // ticket always runs)
        int next = 0;
        if (tid == 0) next = atomicAdd(&sync[0], 1);
        // decode: iterations 0 .. kLag-1 hold y tiles only, then y and z
        // tiles, the last kLag iterations z tiles only
        bool ytile;
        int kx, idx;
        const int64_t head = (int64_t)kLag * nslab;
        const int64_t body = (int64_t)(nkx - kLag) * (nslab + nzt);
        if (t < head) {
            ytile = true;
            kx = (int)(t / nslab);
            idx = (int)(t % nslab);
        } else if (t < head + body) {
            const int64_t u = t - head;
            const int it = kLag + (int)(u / (nslab + nzt));
            const int r = (int)(u % (nslab + nzt));
            ytile = r < nslab;
            kx = ytile ? it : it - kLag;
            idx = ytile ? r : r - nslab;
        } else {
            const int64_t u = t - head - body;
            ytile = false;
            kx = nkx - kLag + (int)(u / nzt);
            idx = (int)(u % nzt);
        }
        float2* rp = ring + (size_t)(kx % kRing) * 2 * plane;
        if (ytile) {
            // ---- y tile: 16 z-lines (z0 ..) of k_x, three components, into the ring.
            // The three 16-line component tiles (contiguous blocks) are all
            // fetched at once by bulk copies, before any wait; each buffer is
            // then that component's exchange buffer, the first also the stash.
            const int z0 = zl + kF * idx;
            const size_t tile = (size_t)N * ((size_t)z0 + (size_t)nz * kx);
            if (tid == 0) {
                tc::fence_async_smem();          // the buffers' earlier use is ordered before the copies
                for (int c = 0; c < 3; ++c) {
                    tc::mbar_expect_tx(&mbar[c], kBytes);
                    tc::bulk_g2s(smem + c * BUF, s0 + (size_t)c * Mh + tile, kBytes, &mbar[c]);
                }
            }
            raise_pending(pend);
            if (kx >= kRing) wait_count(&zdone[kx - kRing], nzt, err);
            const int f1 = tid / X::NT, r1 = tid % X::NT;
            const int f2 = tid % kF, i2 = tid / kF;
            float2* stash = smem;
            float2 o[X::N2];
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                float2* B = smem + c * BUF;
                wait_copy(&mbar[c], (par >> c) & 1u, err);
                float2 v[X::N1];
                if (r1 < X::N2) {
#pragma unroll
                    for (int n1 = 0; n1 < X::N1; ++n1) v[n1] = B[f1 * N + X::N2 * n1 + r1];
                }
                __syncthreads();                 // the staged lines are in registers: B becomes the exchange
                if (r1 < X::N2) fft_step1<N, kF, -1>(v, f1, r1, B, twy);
                __syncthreads();
                if (i2 < X::N1) fft_step2<N, kF, -1>(o, f2, i2, B);
                if (c == 0) {
                    __syncthreads();             // every exchange read done: B becomes the stash
                    if (i2 < X::N1) {
#pragma unroll
                        for (int k2 = 0; k2 < X::N2; ++k2) stash[f2 + (kF + 1) * (i2 + X::N1 * k2)] = o[k2];
                    }
                } else if (c == 1) {
                    if (i2 < X::N1) {
#pragma unroll
                        for (int k2 = 0; k2 < X::N2; ++k2) {
                            const int ky = i2 + X::N1 * k2;
                            const float wy = (ky == N / 2) ? 0.f : wy_scale * (float)signed_bin(ky, N);
                            const float2 w = stash[f2 + (kF + 1) * ky];
                            st_l2hint(rp + (size_t)(z0 + f2) + (size_t)nz * ky,
                                      make_float2(w.x - wy * o[k2].y, w.y + wy * o[k2].x), pout);
                        }
                    }
                } else if (i2 < X::N1) {
#pragma unroll
                    for (int k2 = 0; k2 < X::N2; ++k2)
                        st_l2hint(rp + plane + (size_t)(z0 + f2) + (size_t)nz * (i2 + X::N1 * k2), o[k2], pout);
                }
            }
            par ^= 7u;
            pend = &ydone[kx];
        } else {
            // ---- z tile: 16 k_y lines of k_x from the ring, filter, inverse z, into s1.
            // Both fields' 16-line tiles (contiguous in the ring plane) come
            // in by bulk copies once the y tiles of k_x are done; the proxy
            // fence puts those tiles' generic stores, acquired by thread 0,
            // ahead of the copies.
            raise_pending(pend);
            wait_count(&ydone[kx], nslab, err);
            const int ky0 = kF * idx;
            if (tid == 0) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                tc::fence_async_smem();
                for (int c = 0; c < 2; ++c) {
                    tc::mbar_expect_tx(&mbar[c], kBytes);
                    tc::bulk_g2s(smem + c * BUF, rp + (size_t)c * plane + (size_t)N * ky0, kBytes, &mbar[c]);
                }
            }
            float2* B0 = smem;
            float2* B1 = smem + BUF;
            float2* stash = smem + 2 * BUF;
            const int f = tid / X::NT, r = tid % X::NT;
            wait_copy(&mbar[0], par & 1u, err);
            zstaged_step1<N>(B0, r, f, zl, zh, twz);
            __syncthreads();
            float2 xw[X::N2];
            if (r < X::N1) {
                fft_step2<N, kF, -1>(xw, f, r, B0);
#pragma unroll
                for (int k2 = 0; k2 < X::N2; ++k2) stash[f + (kF + 1) * (r + X::N1 * k2)] = xw[k2];
            }
            wait_copy(&mbar[1], (par >> 1) & 1u, err);
            par ^= 3u;
            zstaged_step1<N>(B1, r, f, zl, zh, twz);
            __syncthreads();
            float2 xh[X::N2];
            if (r < X::N1) fft_step2<N, kF, -1>(xh, f, r, B1);
            __syncthreads();
            if (r < X::N1) {
                const int ky = ky0 + f;
                const float wxd = wx_scale * (float)kx;
                const float wyd = wy_scale * (float)signed_bin(ky, ny);
                const float base = wxd * wxd + wyd * wyd;
#pragma unroll
                for (int k2 = 0; k2 < X::N2; ++k2) {
                    const int kz = r + X::N1 * k2;
                    const float wzd = wz_scale * (float)signed_bin(kz, N);
                    const float wzn = (kz == N / 2) ? 0.f : wzd;
                    const float den = base + wzd * wzd;
                    const float sc = den > 0.f ? inv_m / den : 0.f;
                    const float2 w = stash[f + (kF + 1) * kz];
                    const float2 sv = make_float2(w.x - wzn * xh[k2].y, w.y + wzn * xh[k2].x);
                    xw[k2] = make_float2(sv.x * sc, sv.y * sc);
                }
                fft_step1_swapped<N, kF, +1>(xw, f, r, B1, twz);
            }
            __syncthreads();
            if (r < X::N2) {
                float2 o[X::N1];
                fft_step2_swapped<N, kF, +1>(o, f, r, B1);
                float2* dst = s1 + (size_t)N * ((size_t)(ky0 + f) + (size_t)ny * kx);
#pragma unroll
                for (int k2 = 0; k2 < X::N1; ++k2) st_l2hint(dst + r + X::N2 * k2, o[k2], pout);
            }
            pend = &zdone[kx];
        }
        // two slots: a slot is written again only two barriers after its read
        slot ^= 1;
        if (tid == 0) s_ticket[slot] = next;
        __syncthreads();
        t = s_ticket[slot];
    }
    raise_pending(pend);
}

template <int N>
cudaError_t run_fyz(ftr_ctx* c) {
    using X = Xchg<N, kF>;
    const size_t smem = sizeof(float2) * 3 * YzBuf<N>::value;
    const int threads = kF * X::NT;
    cudaError_t e = ensure_smem(k_fyz<N>, smem, c->device);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fyz<N>, threads, smem)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int nkx = c->g.n[0] / 2 + 1;
    // at most one CTA per tile of a fully live grid
    const int64_t max_tiles = (int64_t)nkx * (N / kF + c->g.n[2] / kF);
    const int grid = (int)(per_sm * sms < max_tiles ? per_sm * sms : max_tiles);
    if ((e = cudaMemsetAsync(c->d_yz_sync, 0, sizeof(int) * (1 + 2 * nkx), c->stream)) != cudaSuccess) return e;
    const double two_pi = 2.0 * 3.14159265358979323846;
    const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
    const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
    const float wz = (float)(two_pi / (c->g.n[2] * c->g.h[2]));
    const float inv_m = (float)(1.0 / (double)c->M);
    const int ring = yz_ring_planes(c->g.n);
    launch_pdl(k_fyz<N>, grid, threads, smem, c->stream, c->g, (const float2*)c->d_s0, c->d_s1, c->d_ring, ring,
               ring / 2, c->Mh,
               (const float2*)c->d_tw[1], (const float2*)c->d_tw[2], wx, wy, wz, inv_m, (const int*)c->d_meta,
               c->d_yz_sync, c->d_kerr);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace

// k_x planes of the ring: about kRingBytes, at least 4, at most every plane
int yz_ring_planes(const int n[3]) {
    const size_t plane = 2 * sizeof(float2) * (size_t)n[1] * n[2];
    const int nkx = n[0] / 2 + 1;
    int r = (int)(kRingBytes / plane);
    if (r < 4) r = 4;
    if (r > nkx) r = nkx;
    return r;
}

cudaError_t fft_yz_init(const float2* w96) { return upload_w96_table(w96); }

bool yz_supported(const int n[3]) {
    if (n[1] != n[2]) return false;
    switch (n[1]) {
        case 64: case 96: case 128: case 192: case 256: case 384: return true;
        default: return false;
    }
}

size_t yz_ring_elems(const int n[3]) { return (size_t)yz_ring_planes(n) * 2 * (size_t)n[1] * n[2]; }

int yz_sync_ints(const int n[3]) { return 1 + 2 * (n[0] / 2 + 1); }

cudaError_t launch_fyz(ftr_ctx* c) {
    if (!yz_supported(c->g.n) || !c->d_ring || !c->d_yz_sync) return cudaErrorInvalidValue;
    switch (c->g.n[1]) {
        case 64: return run_fyz<64>(c);
        case 96: return run_fyz<96>(c);
        case 128: return run_fyz<128>(c);
        case 192: return run_fyz<192>(c);
        case 256: return run_fyz<256>(c);
        case 384: return run_fyz<384>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
