// merge.cu -- exclusive grain association, track order and line fit.
//
// Association (Section 2): "each grain used only once, threshold applied
// again".  The defined result is the sequential greedy pass over candidates
// in key order (count descending, rank lo, rank hi): a candidate keeps its
// unused tube grains and is accepted iff at least min_hits remain.
//
// The device computes exactly that result in rounds.  In a round every
// undecided candidate first counts its unused grains; with fewer than
// min_hits it can never be accepted (its unused set only shrinks), so it is
// rejected.  The others post their key on each unused grain (atomicMin).  A
// candidate holding the minimum key on all its unused grains is "ready": every
// earlier candidate sharing one of those grains is already decided, so its
// unused set is final.  It recounts that set -- a candidate accepted earlier
// in the same phase may have taken some of its grains -- and is accepted iff
// at least min_hits remain, else rejected.  Ready candidates share no unused
// grain, so they mark their grains in parallel.  The lowest undecided key is
// always ready, so every round decides at least one candidate.
//
// Key slots are cleaned by their posters: a candidate decided in phase 2
// resets the slots it holds; one still undecided resets last round's slots of
// all its grains at the start of the next round.
//
// A candidate is only ever blocked by candidates of smaller key, so the
// rounds run over windows of the key-sorted candidate list, one window after
// the other: a window's candidates are decided with every earlier window
// already final and no later one taking part.  The result is the same; a
// candidate joins only the rounds of its own window instead of every round
// until its decision.
//
// Rounds are separated by a grid barrier in one cooperative launch; every
// wait is bounded and a timeout sets ERRB_TIMEOUT instead of hanging.  The
// launch covers the device; a short candidate list keeps only a few of its
// blocks (the result does not depend on how many).
#include "common.cuh"
#include <math.h>

namespace et {

// Device mirror of et_track (include/et.h).
struct TrackOut {
    int seed_i, seed_j, nhits, view;
    long long member_offset;
    float c[3], u[3], tmin, tmax;
    int count, reserved;
};
static_assert(sizeof(TrackOut) == 64, "et_track layout");

namespace {

constexpr int MT = 256;
constexpr unsigned long long BARRIER_SPIN_LIMIT = 1ull << 24;  // x ~128 ns sleep ~ 2 s

__device__ __forceinline__ u32 ld_cg_u32(const u32 *p) { return __ldcg(p); }

// Candidates per block in use: the association keeps one block per MT / 32
// candidates (one candidate per warp, whose dependent loads are the round's
// latency), so a short candidate list runs on few blocks whose barriers are
// cheap, a long one on the whole grid.
constexpr u64 MERGE_CANDS_PER_BLOCK = MT / 32;

__global__ void __launch_bounds__(MT) k_merge(Batch b, Work w) {
    griddep_launch();
    griddep_wait();
    Ctl *ctl = b.ctl;
    if (input_failed(ctl)) return;   // decided before launch: uniform over the grid
    const u64 nc = min(ctl->n_cand, w.cand_cap);
    // blocks in use (uniform: every block read the same count)
    const unsigned nb = (unsigned)min((u64)gridDim.x, max((u64)1, (nc + MERGE_CANDS_PER_BLOCK - 1) / MERGE_CANDS_PER_BLOCK));
    if (blockIdx.x >= nb) return;
    const unsigned long long lim = b.spin_limit > 0 ? (unsigned long long)b.spin_limit : BARRIER_SPIN_LIMIT;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)nb * blockDim.x) >> 5;
    const u32 H = (u32)b.H;
    __shared__ int keep[MT / 32][32];   // per warp: undecided candidates waiting to be appended
    // candidates per window: at least 2^18, at most 128 windows, unless set
    const u64 win = w.window ? w.window : max((u64)1 << 18, (nc + 128 - 1) / 128);
    u32 round = 0;   // counts all rounds: it selects the ping-pong buffers
    for (u64 w0 = 0; w0 < nc; w0 += win) {
    const u64 w1 = min(nc, w0 + win);
    for (u32 wr = 0;; ++wr, ++round) {
        u64 *B = w.best[round & 1];
        u64 *Bp = w.best[(round + 1) & 1];
        // candidates of this round: the window first, then the carried list
        const bool first = wr == 0;
        const int *list = first ? nullptr : w.clist[round & 1];
        const long long nl = first ? (long long)(w1 - w0) : (long long)__ldcg(&ctl->ncl[round & 1]);
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->ncl[(round + 1) & 1] = 0;
        // ---- phase 1: reject hopeless candidates, post keys on unused grains
        u32 my_active = 0;
        for (long long i = gwarp; i < nl; i += nwarps) {
            // lists and states are rewritten by other SMs between rounds: read through L2
            const long long c = list ? __ldcg(&list[i]) : (long long)w.corder[w0 + i];
            if (__ldcg(&w.c_state[c]) != CS_UNDECIDED) continue;
            const u64 m0 = w.c_moff[c], m1 = w.c_moff[c + 1];
            if (m1 - m0 <= 32) {   // one chunk: member and its state stay in registers
                const u64 m = m0 + lane;
                const bool in = m < m1;
                const int g = in ? w.members[m] : 0;
                if (in && !first) Bp[g] = ~0ull;
                const bool fr = in && __ldcg(&w.owner[g]) < 0;
                const u32 nfree = __popc(__ballot_sync(0xffffffffu, fr));
                if (nfree < H) {
                    if (lane == 0) w.c_state[c] = CS_REJECTED;
                    continue;
                }
                if (fr) atomicMin(&B[g], w.c_key[c]);
                ++my_active;
                continue;
            }
            u32 nfree = 0;
            for (u64 base = m0; base < m1; base += 32) {
                const u64 m = base + lane;
                const bool in = m < m1;
                const int g = in ? w.members[m] : 0;
                if (in && !first) Bp[g] = ~0ull;   // entries this candidate posted last round
                const bool fr = in && __ldcg(&w.owner[g]) < 0;
                nfree += __popc(__ballot_sync(0xffffffffu, fr));
            }
            if (nfree < H) {
                if (lane == 0) w.c_state[c] = CS_REJECTED;
                continue;
            }
            const u64 key = w.c_key[c];
            for (u64 base = m0; base < m1; base += 32) {
                const u64 m = base + lane;
                if (m < m1) {
                    const int g = w.members[m];
                    if (__ldcg(&w.owner[g]) < 0) atomicMin(&B[g], key);
                }
            }
            ++my_active;
        }
        if (lane == 0 && my_active) atomicAdd(&ctl->active[round & 1], my_active);
        if (!coop_barrier(ctl->bar, nb, &ctl->error, ERRB_TIMEOUT, lim)) return;
        const u32 active = ld_cg_u32(&ctl->active[round & 1]);
        if (blockIdx.x == 0 && threadIdx.x == 0 && round < 64) ctl->round_active[round] = active;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->active[(round + 1) & 1] = 0;
        if (active == 0) {   // the window is decided (uniform: every block read the same count)
            ++round;
            // the next window's first round counts into the counter just reset
            if (!coop_barrier(ctl->bar, nb, &ctl->error, ERRB_TIMEOUT, lim)) return;
            break;
        }
        // ---- phase 2: accept ready candidates, carry the others to the next round
        int *next = w.clist[(round + 1) & 1];
        u64 *next_n = &ctl->ncl[(round + 1) & 1];
        int nkeep = 0;   // warp-uniform
        for (long long i = gwarp; i < nl; i += nwarps) {
            const long long c = list ? __ldcg(&list[i]) : (long long)w.corder[w0 + i];
            if (__ldcg(&w.c_state[c]) != CS_UNDECIDED) continue;
            const u64 m0 = w.c_moff[c], m1 = w.c_moff[c + 1];
            const u64 key = w.c_key[c];
            if (m1 - m0 <= 32) {   // one chunk: member and its state stay in registers
                const u64 m = m0 + lane;
                const bool in = m < m1;
                const int g = in ? w.members[m] : 0;
                const bool fr = in && __ldcg(&w.owner[g]) < 0;
                const bool bad = fr && __ldcg(&B[g]) != key;
                if (__any_sync(0xffffffffu, bad)) {
                    if (lane == 0) keep[wib][nkeep] = (int)c;
                    if (++nkeep == 32) {
                        __syncwarp();
                        u64 pos = 0;
                        if (lane == 0) pos = atomicAdd(next_n, 32ull);
                        pos = __shfl_sync(0xffffffffu, pos, 0);
                        next[pos + lane] = keep[wib][lane];
                        nkeep = 0;
                        __syncwarp();
                    }
                    continue;
                }
                const u32 nfree = __popc(__ballot_sync(0xffffffffu, fr));
                const bool accept = nfree >= H;
                if (fr) {
                    if (accept) w.owner[g] = (int)c;
                    B[g] = ~0ull;
                }
                if (lane == 0) {
                    w.c_nfree[c] = nfree;
                    w.c_state[c] = accept ? CS_ACCEPTED : CS_REJECTED;
                }
                continue;
            }
            bool ready = true;
            u32 nfree = 0;
            for (u64 base = m0; base < m1; base += 32) {
                const u64 m = base + lane;
                bool fr = false, bad = false;
                if (m < m1) {
                    const int g = w.members[m];
                    fr = __ldcg(&w.owner[g]) < 0;
                    bad = fr && __ldcg(&B[g]) != key;
                }
                if (__any_sync(0xffffffffu, bad)) {
                    ready = false;
                    break;
                }
                nfree += __popc(__ballot_sync(0xffffffffu, fr));
            }
            if (!ready) {
                if (lane == 0) keep[wib][nkeep] = (int)c;
                if (++nkeep == 32) {
                    __syncwarp();
                    u64 pos = 0;
                    if (lane == 0) pos = atomicAdd(next_n, 32ull);
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    next[pos + lane] = keep[wib][lane];
                    nkeep = 0;
                    __syncwarp();
                }
                continue;
            }
            // ready: the unused grains are exactly those where this key is the
            // minimum; nobody else can take them any more
            const bool accept = nfree >= H;
            for (u64 base = m0; base < m1; base += 32) {
                const u64 m = base + lane;
                if (m < m1) {
                    const int g = w.members[m];
                    if (__ldcg(&w.owner[g]) < 0) {
                        if (accept) w.owner[g] = (int)c;
                        B[g] = ~0ull;
                    }
                }
            }
            if (lane == 0) {
                w.c_nfree[c] = nfree;
                w.c_state[c] = accept ? CS_ACCEPTED : CS_REJECTED;
            }
        }
        if (nkeep > 0) {
            __syncwarp();
            u64 pos = 0;
            if (lane == 0) pos = atomicAdd(next_n, (u64)nkeep);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (lane < nkeep) next[pos + lane] = keep[wib][lane];
            __syncwarp();
        }
        if (!coop_barrier(ctl->bar, nb, &ctl->error, ERRB_TIMEOUT, lim)) return;
    }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->rounds = round;
}

// Angle cut (ET_FLAG_ANGLE_CUT): keep a track iff
//     nhits >= cut_base + cut_slope * min(tan theta, cut_tmax),
// tan theta = sqrt(wx^2 + wy^2) / |wz| for the seed vector w, in exact
// integers: with A = nhits - cut_base, keep iff A >= 0 and either
// wx^2 + wy^2 >= cut_tmax^2 wz^2 (tan theta capped) and A >= cut_slope cut_tmax,
// or A^2 wz^2 >= cut_slope^2 (wx^2 + wy^2) (128-bit products).
__device__ __forceinline__ bool angle_cut_keeps(const Batch &b, int4 glo, int4 ghi, long long nhits) {
    const long long A = nhits - b.cut_base;
    if (A < 0) return false;
    const long long wx = ghi.x - glo.x, wy = ghi.y - glo.y, wz = ghi.z - glo.z;
    const unsigned long long t2 = (unsigned long long)(wx * wx + wy * wy), z2 = (unsigned long long)(wz * wz);
    const unsigned long long tm = (unsigned long long)b.cut_tmax, sl = (unsigned long long)b.cut_slope;
    if ((unsigned __int128)t2 >= (unsigned __int128)(tm * tm) * z2) return (unsigned long long)A >= sl * tm;
    return (unsigned __int128)((unsigned long long)A * (unsigned long long)A) * z2 >=
           (unsigned __int128)(sl * sl) * t2;
}

// Single-pass association (ET_FLAG_SINGLE_PASS), step 1: every grain keeps the
// smallest key of the candidates whose tube holds it (one warp per candidate).
__global__ void k_sp_best(Batch b, Work w) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const int lane = threadIdx.x & 31;
    const u64 nw = (u64)gridDim.x * (blockDim.x >> 5);
    for (u64 c = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nc; c += nw) {
        const u64 key = w.c_key[c], m0 = w.c_moff[c], m1 = w.c_moff[c + 1];
        for (u64 m = m0 + lane; m < m1; m += 32) atomicMin(&w.best[0][w.members[m]], key);
    }
}

// Step 2: a candidate owns the grains whose smallest key is its own; it is a
// track iff it owns at least min_hits of them.
__global__ void k_sp_own(Batch b, Work w) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const int lane = threadIdx.x & 31;
    const u64 nw = (u64)gridDim.x * (blockDim.x >> 5);
    for (u64 c = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nc; c += nw) {
        const u64 key = w.c_key[c], m0 = w.c_moff[c], m1 = w.c_moff[c + 1];
        u32 own = 0;
        for (u64 m = m0 + lane; m < m1; m += 32) own += w.best[0][w.members[m]] == key;
        own = __reduce_add_sync(0xffffffffu, own);
        const bool accept = own >= (u32)b.H;
        if (accept)
            for (u64 m = m0 + lane; m < m1; m += 32) {
                const int g = w.members[m];
                if (w.best[0][g] == key) w.owner[g] = (int)c;
            }
        if (lane == 0) {
            w.c_nfree[c] = own;
            w.c_state[c] = accept ? CS_ACCEPTED : CS_REJECTED;
        }
    }
}

// Accepted candidates -> list (any order) with sort keys.
__global__ void k_collect(Batch b, Work w, Out o) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 nc = min(b.ctl->n_cand, w.cand_cap);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
        if (w.c_state[c] != CS_ACCEPTED) continue;
        if ((b.flags & ET_FLAG_ANGLE_CUT) && !angle_cut_keeps(b, b.gr[w.c_lo[c]], b.gr[w.c_hi[c]], w.c_nfree[c]))
            continue;
        const u64 i = atomicAdd(&b.ctl->n_acc, 1ull);
        o.sort_k[0][i] = cand_sort_key(b, w.c_key[c]);
        o.sort_v[0][i] = (u32)c;
    }
}

// After the key sort: second key = view (stable sort keeps key order).
__global__ void k_view_keys(Batch b, Work w, u64 *k, const u32 *v) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;   // a timed-out sort leaves invalid indices
    const u64 na = b.ctl->n_acc;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride)
        k[i] = (u64)view_of(b.goff, b.V, w.c_lo[v[i]]);
}

// Sorted accepted list -> per-track view, nhits (for the member scan) and
// per-view counts (with one view, the view's track offsets).
__global__ void k_track_meta(Batch b, Work w, Out o, const u32 *sorted_c) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 na = b.ctl->n_acc;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < na; t += stride) {
        const u32 c = sorted_c[t];
        o.acc[t] = (int)c;
        const int v = view_of(b.goff, b.V, w.c_lo[c]);
        o.trk_view[t] = v;
        o.trk_moff[t] = w.c_nfree[c];
        if (b.V > 1) atomicAdd((unsigned long long *)&o.view_trk[v], 1ull);
    }
    if (b.V == 1 && blockIdx.x == 0 && threadIdx.x == 0) {   // one view: its track offsets directly
        o.view_trk[0] = 0;
        o.view_trk[1] = (long long)na;
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

__device__ __forceinline__ float i128_to_float(__int128 x) {
    const bool neg = x < 0;
    unsigned __int128 m = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const double hi = (double)(unsigned long long)(m >> 64);
    const double lo = (double)(unsigned long long)m;
    const double d = hi * 18446744073709551616.0 + lo;
    return (float)(neg ? -d : d);
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Matrix Computations, Sec. 8.5), FP32.  Columns of V are eigenvectors.
__device__ void jacobi3f(float A[3][3], float V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 12; ++sweep) {
        const float off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const float dg = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0f || off <= 1e-16f * dg) break;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int p = m < 2 ? 0 : 1, q = m < 1 ? 1 : 2;
            if (A[p][q] == 0.0f) continue;
            const float tau = (A[q][q] - A[p][p]) / (2.0f * A[p][q]);
            const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
            const float c = 1.0f / sqrtf(1.0f + t * t), s = t * c;
            for (int k = 0; k < 3; ++k) {
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
}

// One warp per accepted track: exact integer moments about the lo seed grain,
// FP32 principal axis, member projections; member keys for the final sort.
__global__ void k_fit(Batch b, Work w, Out o) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 na = b.ctl->n_acc;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    TrackOut *tracks = (TrackOut *)o.tracks;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < (long long)na; t += nw) {
        const int c = o.acc[t];
        const int lo = w.c_lo[c], hi = w.c_hi[c];
        const int4 ga = b.gr[lo], gb = b.gr[hi];
        const u64 m0 = w.c_moff[c], m1 = w.c_moff[c + 1];
        const u64 obase = o.trk_moff[t];
        long long s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0};
        u32 written = 0;
        for (u64 base = m0; base < m1; base += 32) {
            const u64 m = base + lane;
            int g = -1;
            if (m < m1) g = w.members[m];
            const bool own = g >= 0 && w.owner[g] == c;
            const unsigned bal = __ballot_sync(0xffffffffu, own);
            if (own) {
                const int4 p = b.gr[g];
                const long long dx = p.x - ga.x, dy = p.y - ga.y, dz = p.z - ga.z;
                s1[0] += dx; s1[1] += dy; s1[2] += dz;
                s2[0] += dx * dx; s2[1] += dy * dy; s2[2] += dz * dz;
                s2[3] += dx * dy; s2[4] += dx * dz; s2[5] += dy * dz;
                const u64 pos = obase + written + __popc(bal & ((1u << lane) - 1u));
                o.sort_k[0][pos] = ((u64)t << b.rbits) | (u64)p.w;
                o.sort_v[0][pos] = 0u;
            }
            written += __popc(bal);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) s1[k] = warp_sum_ll(s1[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) s2[k] = warp_sum_ll(s2[k]);
        const long long n = (long long)written;
        // scatter matrix times n^2 ... exact: M_ab = n S2_ab - S1_a S1_b
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        float cov[6];
        const float inv_n2 = 1.0f / ((float)n * (float)n);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const __int128 M = (__int128)n * s2[k] - (__int128)s1[ia[k]] * s1[ib[k]];
            cov[k] = i128_to_float(M) * inv_n2;
        }
        float A[3][3] = {{cov[0], cov[3], cov[4]}, {cov[3], cov[1], cov[5]}, {cov[4], cov[5], cov[2]}};
        float V[3][3];
        jacobi3f(A, V);
        int best = 0;
        if (A[1][1] > A[best][best]) best = 1;
        if (A[2][2] > A[best][best]) best = 2;
        float u[3] = {V[0][best], V[1][best], V[2][best]};
        const float nrm = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        u[0] /= nrm; u[1] /= nrm; u[2] /= nrm;
        const float dot = u[0] * (float)(gb.x - ga.x) + u[1] * (float)(gb.y - ga.y) + u[2] * (float)(gb.z - ga.z);
        bool flip = dot < 0.0f;
        if (dot == 0.0f) flip = (u[0] != 0.0f) ? u[0] < 0.0f : ((u[1] != 0.0f) ? u[1] < 0.0f : u[2] < 0.0f);
        if (flip) { u[0] = -u[0]; u[1] = -u[1]; u[2] = -u[2]; }
        // centroid relative to the lo grain.  A member's offset from the
        // centroid, times n, is the exact integer n d - S1 (d its offset from
        // the lo grain), so a projection's rounding scales with the
        // projection itself, not with the view or the track length
        const float fn = (float)n;
        const float ca[3] = {(float)s1[0] / fn, (float)s1[1] / fn, (float)s1[2] / fn};
        const float cen[3] = {(float)ga.x + ca[0], (float)ga.y + ca[1], (float)ga.z + ca[2]};
        float tmin = 3.0e38f, tmax = -3.0e38f;
        for (u64 base = m0; base < m1; base += 32) {
            const u64 m = base + lane;
            if (m < m1) {
                const int g = w.members[m];
                if (w.owner[g] == c) {
                    const int4 p = b.gr[g];
                    const long long ex = n * (long long)(p.x - ga.x) - s1[0];
                    const long long ey = n * (long long)(p.y - ga.y) - s1[1];
                    const long long ez = n * (long long)(p.z - ga.z) - s1[2];
                    const float tt = ((float)ex * u[0] + (float)ey * u[1] + (float)ez * u[2]) / fn;
                    tmin = fminf(tmin, tt);
                    tmax = fmaxf(tmax, tt);
                }
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, s));
            tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, s));
        }
        if (lane == 0) {
            TrackOut r;
            r.seed_i = ga.w;
            r.seed_j = gb.w;
            r.nhits = (int)n;
            r.view = o.trk_view[t];
            r.member_offset = (long long)obase;
            r.c[0] = cen[0]; r.c[1] = cen[1]; r.c[2] = cen[2];
            r.u[0] = u[0]; r.u[1] = u[1]; r.u[2] = u[2];
            r.tmin = tmin;
            r.tmax = tmax;
            r.count = (int)w.c_cnt[c];
            r.reserved = 0;
            tracks[t] = r;
        }
    }
}

__global__ void k_members_out(Batch b, Out o, const u64 *sorted_k) {
    griddep_launch();
    griddep_wait();
    if (input_failed(b.ctl)) return;
    const u64 nm = b.ctl->n_out_members;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += stride)
        o.out_members[i] = (int)(sorted_k[i] & ((1ull << b.rbits) - 1ull));
}

unsigned sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return (unsigned)sms;
}

int bits_for(unsigned long long maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

}  // namespace

int merge_grid_blocks(int device) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge, MT, 0);
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_merge_coop(const Batch &b, const Work &w, int grid, cudaStream_t st) {
    Batch bb = b;
    Work ww = w;
    void *args[] = {&bb, &ww};
    return cudaLaunchCooperativeKernel((const void *)k_merge, dim3(grid), dim3(MT), args, 0, st);
}

const u32 *launch_cand_order(const Batch &b, const Work &w, Out &o, void *temp, cudaStream_t st) {
    const int cur = radix_sort_pairs_dev(o.sort_k[0], o.sort_v[0], o.sort_k[1], o.sort_v[1], (long long)o.acc_cap,
                                         &b.ctl->n_cand, 3 * b.rbits, temp, st, &b.ctl->error, ERRB_TIMEOUT,
                                         b.ctl->bar, b.spin_limit);
    return o.sort_v[cur];
}

void launch_single_pass(const Batch &b, const Work &w, cudaStream_t st) {
    const unsigned g = sm_count() * 8;
    launch_dep(k_sp_best, dim3(g), dim3(256), 0, st, b, w);
    launch_dep(k_sp_own, dim3(g), dim3(256), 0, st, b, w);
}

// Accepted list sorted by (view, key); per-view track offsets; member offsets;
// fit; members sorted within each track.  acc_cap and member_cap size the
// launches; the device counters decide the work.
void launch_output(const Batch &b, const Work &w, Out &o, long long acc_cap, long long out_member_cap,
                   void *temp, cudaStream_t st) {
    const unsigned g = sm_count() * 4;
    launch_dep(k_collect, dim3(g), dim3(256), 0, st, b, w, o);
    u64 *na = &b.ctl->n_acc;
    int cur = radix_sort_pairs_dev(o.sort_k[0], o.sort_v[0], o.sort_k[1], o.sort_v[1], acc_cap, na, 3 * b.rbits,
                                   temp, st, &b.ctl->error, ERRB_TIMEOUT, b.ctl->bar, b.spin_limit);
    if (b.V > 1) {
        launch_dep(k_view_keys, dim3(g), dim3(256), 0, st, b, w, o.sort_k[cur], o.sort_v[cur]);
        int c2 = radix_sort_pairs_dev(o.sort_k[cur], o.sort_v[cur], o.sort_k[cur ^ 1], o.sort_v[cur ^ 1], acc_cap,
                                      na, bits_for((unsigned long long)(b.V - 1)), temp, st, &b.ctl->error, ERRB_TIMEOUT,
                                      b.ctl->bar, b.spin_limit);
        cur = c2 ? (cur ^ 1) : cur;
    }
    if (b.V > 1) cudaMemsetAsync(o.view_trk, 0, sizeof(long long) * (b.V + 1), st);
    launch_dep(k_track_meta, dim3(g), dim3(256), 0, st, b, w, o, o.sort_v[cur]);
    if (b.V > 1)
        exclusive_scan_u64_dev((const u64 *)o.view_trk, (u64 *)o.view_trk, b.V, nullptr, temp, nullptr, st,
                               &b.ctl->error, ERRB_TIMEOUT, b.ctl->bar, b.spin_limit);
    exclusive_scan_u64_dev(o.trk_moff, o.trk_moff, acc_cap, na, temp, &b.ctl->n_out_members, st, &b.ctl->error,
                           ERRB_TIMEOUT, b.ctl->bar, b.spin_limit);
    launch_dep(k_fit, dim3(g), dim3(256), 0, st, b, w, o);
    const int tbits = bits_for((unsigned long long)(acc_cap > 0 ? acc_cap : 1));
    int cm = radix_sort_pairs_dev(o.sort_k[0], o.sort_v[0], o.sort_k[1], o.sort_v[1], out_member_cap,
                                  &b.ctl->n_out_members, b.rbits + tbits, temp, st, &b.ctl->error, ERRB_TIMEOUT,
                                  b.ctl->bar, b.spin_limit);
    launch_dep(k_members_out, dim3(g), dim3(256), 0, st, b, o, o.sort_k[cm]);
}

}  // namespace et
