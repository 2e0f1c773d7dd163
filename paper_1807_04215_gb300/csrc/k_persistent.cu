// Persistent work-queue kernel: the recursion of several plans, whose grid
// sizes may differ, in one launch.
//
// The host (api.cpp) records every launch that gridspt_run_orders would make
// for each plan as a stage (a pass over tiles: column blocks, z row groups,
// cell blocks) and lays the stages of all plans out in one queue in an order
// that respects each plan's chain (a stage waits only for its predecessor in
// its own chain). The kernel is launched with as many 256-thread blocks as
// fit on the GPU at once. Each block takes the next ticket from a global
// counter, maps it to (stage, tile), waits until the stage's predecessor has
// counted all its tiles done, runs the tile with the same per-element
// arithmetic as the pass's own kernel, and counts the tile done.
//
// Progress: a block waits only for tiles with smaller tickets, and a ticket is
// only taken by a block that is running, so every wait ends once earlier
// tiles finish, whatever the number of resident blocks. Every wait is also
// bounded in time (wait_ns of the global timer): when it runs out the block
// sets the plan's status word (kStatusWaitQueue, reported by gridspt_check as
// GRIDSPT_E_TIMEOUT) and an abort flag, and every block returns at its next
// ticket or wait. Nothing traps or spins without limit.
//
// Memory ordering: a finished tile's stores are ordered before its done count
// by a block barrier and a GPU-scope fence; the waiting block's thread 0
// reads the count with acquire semantics and a block barrier orders the other
// threads' loads after it. Fields written earlier in the launch are read with
// ordinary (coherent) loads, never through the read-only data path.
//
// Tile bodies: the column passes (x expansion, y expansion, forward column
// passes) run the bodies of k_transform.cuh with tile widths that give 256
// threads; the z passes run the warp-row body of k_zrow (one row group per
// warp) for power-of-two N, and for N = 3 * 2^a a warp-row form that reads the
// partner fields straight from global memory instead of staging them in
// shared memory (their staged rows would not fit twice per SM); the diagonal
// pairs run product_cells. Accumulation
// orders and transform arithmetic are those of the separate kernels, so the
// results are bitwise equal to gridspt_run_orders.
#include "k_transform.cuh"
#include "product_core.cuh"

namespace gridspt {

namespace {

// Warp-row geometry of the queue's z passes (any row length M = N / 2 with
// P = M / E <= 32 lanes per row and 32 % P == 0).
template <int N>
struct QRow {
    static constexpr int M = N / 2, E = fft_elems(M), P = M / E;
    static_assert(P <= 32 && 32 % P == 0, "rows must tile a warp");
    static constexpr int RW = 32 / P;                         // rows per warp
    static constexpr int XROW = M + (M >> 4);                 // padded exchange row
    static constexpr int NTW = fft_row_tw_total<M>();
    static constexpr int HDR = ((NTW + E) * P + 1) / 2 * 2;   // twiddle tables, 16-byte multiple
    static constexpr int WIN = RW * M;                        // input rows of a warp
    static_assert(WIN % 64 == 0, "16-byte row copies by 32 lanes");
    static constexpr int WSTRIDE = WIN + RW * XROW;
    static constexpr size_t smem = sizeof(float2) * (HDR + (size_t)(kQueueThreads / 32) * WSTRIDE);
};

// tile width of the column passes with 256 threads
template <int N>
__host__ __device__ constexpr int qtz() { return kQueueThreads / (N / fft_elems(N)); }

template <int N>
__host__ __device__ constexpr size_t col_smem() {
    return ColSm<N, qtz<N>()>::bytes > colpass_smem<N, qtz<N>()>() ? ColSm<N, qtz<N>()>::bytes
                                                                    : colpass_smem<N, qtz<N>()>();
}

template <int N>
__device__ __forceinline__ void q_tables(float2* twl, float2* twp, const float2* __restrict__ twg) {
    using C = QRow<N>;
    if (threadIdx.x < C::P) {
        fft_row_twiddles<C::M, N>(twl, twg, threadIdx.x);
#pragma unroll
        for (int i = 0; i < C::E; ++i) twp[i * C::P + threadIdx.x] = twg[threadIdx.x + C::P * i];
    }
    __syncthreads();
}

// z expansion (NT = 0: store only; NT = 1, 2: fused pair products of k_zrow),
// one group of RW rows per warp, 8 groups per tile.
template <int N, int NT, bool BAND>
__device__ void q_zrow(const ZPairArgs& args, const float2* __restrict__ twg, float kF, long long tile,
                       float2* sm, bool table_ready) {
    using C = QRow<N>;
    constexpr int M = C::M, E = C::E, P = C::P, RW = C::RW, WIN = C::WIN;
    constexpr int NA = NT > 0 ? NT : 1;
    float2* twl = sm;
    float2* twp = twl + C::NTW * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / P, p = lane - r * P;
    if (!table_ready) q_tables<N>(twl, twp, twg);
    float2* wbase = sm + C::HDR + warp * C::WSTRIDE;
    float2* xrow = wbase + WIN + r * C::XROW;
    const YZExpArgs& z = args.z;
    const int B = BAND ? z.band : 0;
    unsigned inb = 0;            // bit u: this lane's 16-byte piece u of a row window lies at kz < B
#pragma unroll
    for (int u = 0; u < WIN / 64; ++u)
        if (B <= 0 || (2 * (lane + 32 * u)) % M < B) inb |= 1u << u;
    const long long groups = (long long)N * N / RW;
    const long long grp = tile * (kQueueThreads / 32) + warp;
    if (grp >= groups) return;   // no block barrier follows
    const long long fstride2 = args.cells / 2;
    const long long row0 = grp * RW, row = row0 + r;
    float2 accA[NA][E], accB[NA][E];
#pragma unroll
    for (int t = 0; t < NA; ++t)
#pragma unroll
        for (int i = 0; i < E; ++i) accA[t][i] = accB[t][i] = make_float2(0.f, 0.f);
    int cur = -1;
    for (int f = 0; f < z.nout; ++f) {
        const int code = z.codes[f];
        const int in = code & 255, g = (code >> 8) & 3, cc = (code >> 12) & 3, slot = code >> 16;
        if (in != cur) {
            __syncwarp();                                  // earlier reads of the input rows are done
            const float4* src = reinterpret_cast<const float4*>(z.in + in * z.in_stride + row0 * M);
            float4 v[WIN / 64];
#pragma unroll
            for (int u = 0; u < WIN / 64; ++u)
                v[u] = ((inb >> u) & 1u) ? src[lane + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < WIN / 64; ++u) reinterpret_cast<float4*>(wbase)[lane + 32 * u] = v[u];
            __syncwarp();
            cur = in;
        }
        const float2* colp = wbase + r * M;
        float2 x[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = p + P * i;
            float2 Xk = colp[k];
            float2 Xm = k ? colp[M - k] : make_float2(0.f, 0.f);
            if (g) {
                const float k1 = kF * (float)k, k2 = kF * (float)(M - k);
                Xk = cscale(Xk, g == 1 ? k1 : k1 * k1);
                Xm = cscale(Xm, g == 1 ? k2 : k2 * k2);
            }
            if (cc == 1) {
                Xk = cmul_i<+1>(Xk);
                Xm = cmul_i<+1>(Xm);
            } else if (cc == 2) {
                Xk = cmul_i<-1>(Xk);
                Xm = cmul_i<-1>(Xm);
            }
            Xm = cconj(Xm);
            const float2 Ev = cadd(Xk, Xm);
            const float2 Ov = cmul(csub(Xk, Xm), twp[i * P + p]);
            x[i] = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
        }
        fft_row<M, +1>(x, p, xrow, twl);                  // x[i]: real cells 2n, 2n + 1, n = p + P i
        float2* dst = NT > 0 ? (args.store ? reinterpret_cast<float2*>(args.store) + slot * fstride2 : nullptr)
                             : z.out + slot * z.out_stride;
        if (dst) {
#pragma unroll
            for (int i = 0; i < E; ++i) dst[row * M + p + P * i] = x[i];
        }
        if constexpr (NT > 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (t >= args.ntargets) break;
                const PairTarget& T = args.t[t];
                for (int q = 0; q < T.pcount[slot]; ++q) {
                    const float ca = T.pcoef_a[slot][q], cb = T.pcoef_b[slot][q];
                    const bool sq = T.pfield[slot][q] < 0;                    // a square
                    const float2* pr = reinterpret_cast<const float2*>(T.partner) +
                                       (long long)(sq ? 0 : T.pfield[slot][q]) * fstride2 + row * M;
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const float2 gv = sq ? x[i] : pr[p + P * i];
                        const float2 fg = lmul(x[i], gv);
                        accA[t][i] = lfma(ca, fg, accA[t][i]);
                        accB[t][i] = lfma(cb, fg, accB[t][i]);
                    }
                }
            }
        }
    }
    if constexpr (NT > 0) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t >= args.ntargets) break;
            const PairTarget& T = args.t[t];
            if (T.acc_in_a) {
                const float2* ia = reinterpret_cast<const float2*>(T.acc_in_a) + row * M;
                const float2* ib = reinterpret_cast<const float2*>(T.acc_in_b) + row * M;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const float2 va = ia[p + P * i], vb = ib[p + P * i];
                    accA[t][i] = cadd(accA[t][i], va);
                    accB[t][i] = cadd(accB[t][i], vb);
                }
            }
            float2* oa = reinterpret_cast<float2*>(T.out_a) + row * M;
            float2* ob = reinterpret_cast<float2*>(T.out_b) + row * M;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                oa[p + P * i] = lfma(T.ca0, accA[t][i], cscale(accB[t][i], T.ca1));
                ob[p + P * i] = lfma(T.cb0, accA[t][i], cscale(accB[t][i], T.cb1));
            }
        }
    }
}

// Contiguous-axis forward transform of k_zrow_r2c, one row group per warp.
template <int N>
__device__ void q_zr2c(const QStage& st, long long tile, float2* sm, bool table_ready) {
    using C = QRow<N>;
    constexpr int M = C::M, E = C::E, P = C::P, RW = C::RW;
    float2* twl = sm;
    float2* twp = twl + C::NTW * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / P, p = lane - r * P;
    if (!table_ready) q_tables<N>(twl, twp, st.tw);
    float2* xrow = sm + C::HDR + warp * C::WSTRIDE + C::WIN + r * C::XROW;
    const long long per = (long long)N * N / RW;
    const long long grp = tile * (kQueueThreads / 32) + warp;
    if (grp >= per * st.count) return;
    const float half = 0.5f * st.scale;
    const long long fld = grp / per, row = (grp - fld * per) * RW + r;
    const float2* src = st.data + fld * st.fstride + row * M;
    float2* dst = st.data + fld * st.fstride + row * M;
    float2 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = src[p + P * i];
    fft_row<M, -1>(x, p, xrow, twl);
#pragma unroll
    for (int i = 0; i < E; ++i) xrow[xpad(p + P * i)] = x[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = p + P * i;
        const float2 Z = xrow[xpad(k)];
        const float2 Zr = cconj(xrow[xpad(k ? M - k : 0)]);
        const float2 S = cadd(Z, Zr);
        const float2 t = cmul(cconj(twp[i * P + p]), csub(Z, Zr));
        dst[k] = make_float2(half * (S.x + t.y), half * (S.y - t.x));
    }
}

// Layout class of the table a stage kind keeps at the start of shared memory:
// 1 the stage-twiddle table of the expansion column transforms (fft_col),
// 2 the warp-row tables of k_zrow, 3 the warp-row tables of QRow, 4 the table
// of N-th roots of the forward column passes (0: none).
__host__ __device__ constexpr int q_table_class(int kind, bool row_ok) {
    return (kind == Q_XEXP0 || kind == Q_XEXP1 || kind == Q_YEXP) ? 1
           : (kind == Q_COLY || kind == Q_COLX) ? 4
           : kind == Q_Z ? (row_ok ? 2 : 3) : kind == Q_ZR2C ? 3 : 0;
}

template <int N>
__device__ void q_tile(const QStage& st, long long tile, float2* sm, bool tr) {
    constexpr int TZ = qtz<N>();
    const int bx = (int)(tile % st.gx);
    const long long rest = tile / st.gx;
    const int by = (int)(rest % st.gy);
    const int bz = (int)(rest / st.gy);
    switch (st.kind) {
        case Q_XEXP0: xexp_body<N, TZ, 0>(st.x, st.tw, st.kF, st.inv_kF2, bx, by, sm, tr); break;
        case Q_XEXP1: xexp_body<N, TZ, 1>(st.x, st.tw, st.kF, st.inv_kF2, bx, by, sm, tr); break;
        case Q_YEXP: yexp_body<N, TZ, false>(st.y, st.tw, st.kF, bx, by, sm, tr); break;
        case Q_COLY: colpass_body<N, TZ, 1, false>(st.data, st.fstride, st.tw, -1, 0, 0, bx, by, bz, sm, tr); break;
        case Q_COLX:
            colpass_body<N, TZ, 0, true>(st.data, st.fstride, st.tw, st.s2, st.zero_k0, 0, bx, by, bz, sm, tr);
            break;
        case Q_ZR2C: q_zr2c<N>(st, tile, sm, tr); break;
        case Q_Z: {
            const bool band = st.z.z.band > 0;
            if constexpr (RowCfg<N>::ok) {   // power-of-two rows: the z pass of k_zrow (staged partners, prefetch)
                constexpr long long one = 1LL << 40;   // a stride past every group: one group per warp
                const long long g0 = tile * (kQueueThreads / 32);
                if (st.z.ntargets == 0) {
                    if (band) zrow_body<N, 0, true>(st.z, st.tw, st.kF, g0, one, sm, tr);
                    else zrow_body<N, 0, false>(st.z, st.tw, st.kF, g0, one, sm, tr);
                } else if (st.z.ntargets == 1) {
                    if (band) zrow_body<N, 1, true>(st.z, st.tw, st.kF, g0, one, sm, tr);
                    else zrow_body<N, 1, false>(st.z, st.tw, st.kF, g0, one, sm, tr);
                } else {
                    if (band) zrow_body<N, 2, true>(st.z, st.tw, st.kF, g0, one, sm, tr);
                    else zrow_body<N, 2, false>(st.z, st.tw, st.kF, g0, one, sm, tr);
                }
                break;
            }
            // N = 3 * 2^a: one target per stage (the host splits two-target
            // launches), which keeps the accumulators of 12-element rows in registers
            if (st.z.ntargets == 0) {
                if (band) q_zrow<N, 0, true>(st.z, st.tw, st.kF, tile, sm, tr);
                else q_zrow<N, 0, false>(st.z, st.tw, st.kF, tile, sm, tr);
            } else {
                if (band) q_zrow<N, 1, true>(st.z, st.tw, st.kF, tile, sm, tr);
                else q_zrow<N, 1, false>(st.z, st.tw, st.kF, tile, sm, tr);
            }
            break;
        }
        default: break;
    }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// hdr: [0..1] ticket counter (64-bit), [2] abort flag, [3] unused, [4 + s] done tickets of stage s.
// A ticket covers `chunk` consecutive tiles of its stage. Thread 0 takes the
// block's next ticket while the current one runs (the atomic's latency is
// hidden); a block that has seen a stage complete remembers it (a bit per
// stage in shared memory) and does not read its counter again.
constexpr int kQueueBitStages = 8192;

__global__ void __launch_bounds__(kQueueThreads, 2)
k_queue(const QStage* __restrict__ stages, const long long* __restrict__ starts, int nst, long long total,
        int* __restrict__ hdr, int* __restrict__ status, long long wait_ns) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ long long s_ticket;
    __shared__ int s_stage, s_abort;
    __shared__ unsigned s_seen[kQueueBitStages / 32];   // stages this block has seen complete
    __shared__ int s_tabkey;                            // layout class and N of the table in sm (0: none)
    unsigned long long* next = reinterpret_cast<unsigned long long*>(hdr);
    int* abort_flag = hdr + 2;
    int* done = hdr + 4;
    for (int i = threadIdx.x; i < kQueueBitStages / 32; i += blockDim.x) s_seen[i] = 0u;
    if (threadIdx.x == 0) s_tabkey = 0;
    __syncthreads();
    long long t_next = 0;
    if (threadIdx.x == 0) t_next = (long long)atomicAdd(next, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = t_next;
            int ab = *reinterpret_cast<volatile int*>(abort_flag);
            int s = -1;
            if (t < total && !ab) {
                t_next = (long long)atomicAdd(next, 1ull);    // used at the next iteration
                int lo = 0, hi = nst;                          // starts[lo] <= t < starts[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(starts + mid) <= t) lo = mid; else hi = mid;
                }
                s = lo;
                const int dep = __ldg(&stages[s].dep);
                const bool known = dep < kQueueBitStages && dep >= 0 && ((s_seen[dep >> 5] >> (dep & 31)) & 1u);
                if (dep >= 0 && !known) {                      // bounded wait for the predecessor stage
                    const int need = (int)(__ldg(starts + dep + 1) - __ldg(starts + dep));
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire(done + dep) < need) {
                        if (*reinterpret_cast<volatile int*>(abort_flag)) { ab = 1; break; }
                        if (global_ns() - t0 > (unsigned long long)wait_ns) {
                            atomicOr(status, kStatusWaitQueue);
                            atomicExch(abort_flag, 1);
                            ab = 1;
                            break;
                        }
                        __nanosleep(100);
                    }
                    if (!ab && dep < kQueueBitStages) s_seen[dep >> 5] |= 1u << (dep & 31);
                }
            }
            s_ticket = t;
            s_stage = s;
            s_abort = ab || s < 0;
        }
        __syncthreads();
        if (s_abort) return;
        const int s = s_stage;
        const QStage& st = stages[s];
        const long long first = (s_ticket - starts[s]) * st.chunk;
        const long long last = first + st.chunk < st.ntiles ? first + st.chunk : st.ntiles;
        for (long long tile = first; tile < last; ++tile) {
            if (st.kind == Q_PRODUCT) {
                const long long i = tile * kQueueThreads + threadIdx.x;
                if (i < st.pr.cells / 4) product_cells(st.pr, i, PlainLoad{});
            } else if (st.kind == Q_ZEROBAND) {
                const int Nn = st.N, H = Nn / 4, band = st.band;
                const long long pairs = (long long)Nn * Nn * H;
                const long long j = tile * kQueueThreads + threadIdx.x;
                if (j < 2 * pairs) {
                    const int fld = (int)(j / pairs);
                    const long long i2 = j - fld * pairs;
                    const long long row = i2 / H;
                    const int kz = (int)(2 * (i2 - row * H));
                    const int ky = (int)(row % Nn);
                    if (!(kz < band && (ky < band || ky > Nn - band)))
                        reinterpret_cast<float4*>(fld ? st.data2 : st.data)[i2] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
                const int cls = q_table_class(st.kind, (st.N & (st.N - 1)) == 0);
                const int key = cls ? (cls << 16) | st.N : 0;
                const bool tr = key != 0 && s_tabkey == key;
                switch (st.N) {
                    case 64: q_tile<64>(st, tile, sm, tr); break;
                    case 96: q_tile<96>(st, tile, sm, tr); break;
                    case 128: q_tile<128>(st, tile, sm, tr); break;
                    case 192: q_tile<192>(st, tile, sm, tr); break;
                    case 256: q_tile<256>(st, tile, sm, tr); break;
                    default: break;
                }
                __syncthreads();                          // every thread has read s_tabkey
                if (threadIdx.x == 0) s_tabkey = key;
            }
            __syncthreads();                              // shared buffers free, every store issued
        }
        if (threadIdx.x == 0) {
            __threadfence();                              // the ticket's stores are visible before the count
            if (!st.nosignal) atomicAdd(done + s, 1);
        }
    }
}

template <int N>
constexpr size_t q_smem_n() {
    constexpr size_t z = RowCfg<N>::ok ? RowCfg<N>::smem(2) : QRow<N>::smem;
    return z > col_smem<N>() ? z : col_smem<N>();
}

}  // namespace

bool queue_supported_n(int N) { return N == 64 || N == 96 || N == 128 || N == 192 || N == 256; }

size_t queue_smem_bytes() {
    size_t b = q_smem_n<64>();
    b = q_smem_n<96>() > b ? q_smem_n<96>() : b;
    b = q_smem_n<128>() > b ? q_smem_n<128>() : b;
    b = q_smem_n<192>() > b ? q_smem_n<192>() : b;
    b = q_smem_n<256>() > b ? q_smem_n<256>() : b;
    return b;
}

namespace {
template <int N>
void tiles_n(QStage& st) {
    constexpr int M = N / 2, TZ = qtz<N>();
    constexpr int RW = QRow<N>::RW;
    const long long W = kQueueThreads / 32;
    st.gx = 1;
    st.gy = 1;
    switch (st.kind) {
        case Q_XEXP0:
        case Q_XEXP1: {
            const int B = st.x.band > 0 && st.x.band < M ? st.x.band : 0;
            st.gx = ((B ? B : M) + TZ - 1) / TZ;
            st.gy = B ? 2 * B - 1 : N;
            st.ntiles = (long long)st.gx * st.gy;
            break;
        }
        case Q_YEXP: {
            const int B = st.y.band > 0 && st.y.band < M ? st.y.band : 0;
            st.gx = ((B ? B : M) + TZ - 1) / TZ;
            st.gy = N;
            st.ntiles = (long long)st.gx * st.gy;
            break;
        }
        case Q_COLY:
        case Q_COLX:
            st.gx = (M + TZ - 1) / TZ;
            st.gy = N;
            st.ntiles = (long long)st.gx * st.gy * st.count;
            break;
        case Q_ZR2C:
            st.ntiles = ((long long)N * N / RW * st.count + W - 1) / W;
            break;
        case Q_Z:
            st.ntiles = ((long long)N * N / RW + W - 1) / W;
            break;
        case Q_PRODUCT:
            st.ntiles = (st.pr.cells / 4 + kQueueThreads - 1) / kQueueThreads;
            break;
        case Q_ZEROBAND:
            st.ntiles = (2LL * N * N * (N / 4) + kQueueThreads - 1) / kQueueThreads;
            break;
        default: st.ntiles = 0;
    }
}
}  // namespace

void queue_tiles(QStage& st) {
    st.chunk = 1;
    switch (st.N) {
        case 64: tiles_n<64>(st); break;
        case 96: tiles_n<96>(st); break;
        case 128: tiles_n<128>(st); break;
        case 192: tiles_n<192>(st); break;
        case 256: tiles_n<256>(st); break;
        default: st.ntiles = 0;
    }
}

cudaError_t launch_queue(const QStage* stages, const long long* starts, int nst, long long total, int* hdr,
                         int* status, long long wait_ns, cudaStream_t s) {
    const size_t smem = queue_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_queue, kQueueThreads, smem)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(hdr, 0, sizeof(int) * (4 + (size_t)nst), s)) != cudaSuccess) return e;
    const long long resident = (long long)(per > 0 ? per : 1) * sms;
    const long long grid = total < resident ? (total > 0 ? total : 1) : resident;
    k_queue<<<(unsigned)grid, kQueueThreads, smem, s>>>(stages, starts, nst, total, hdr, status, wait_ns);
    return cudaGetLastError();
}

}  // namespace gridspt
