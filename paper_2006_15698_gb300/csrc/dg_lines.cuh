// dg_lines.cuh -- the float form's single-mesh RK stage as a z-marching
// column kernel with one thread per z node line.  Included by dg_kernels.cuh
// (inside namespace dg), after dg_column.cuh, whose slot layout, prefetch,
// traces and flux routines it shares.
//
// As in column_stage_kernel, a CTA walks a column of TX x TY elements up a
// chunk of z layers and the layers ahead are staged in a ring of shared-
// memory slots by cp.async.  Here a thread owns the N nodes
// (i, j, 0..N-1) of one element of the layer, so all work along z stays in
// its registers: the z fluxes of its nodes and their weak z-derivative, the
// traces at the two z ends of its line and the z interface flux above it
// (kept as the next layer's -z face flux).  Per layer:
//
//   P  every thread: Euler fluxes (Eq. 2-3) of its nodes, x and y fluxes ->
//      shared memory as x and y node lines; the z interface flux above its
//      line (local Lax-Friedrichs, Sec. II.B) from its own +z trace and the
//      -z trace of the line above in the next slot;
//      interface tasks: the local Lax-Friedrichs flux at every x and y face
//      point of the layer, each interface once, from the traces of the
//      staged node lines on both sides (a neighbour column's line read
//      through L2) -> shared memory
//   G  every thread: weak derivative, lift of the six face fluxes and the
//      stage update of its nodes -> DRAM
//
// Traces, interface fluxes, node fluxes, the derivative sums and the update
// use the same functions in the same operation order as column_stage_kernel,
// so the two kernels give the same floats.
#pragma once

// Column cross-sections per N (= p + 1): one thread per z line, 64 to 256
// threads per CTA (measured on GB300; wider ones lose occupancy to shared
// memory and registers).  NS: slots in the ring of staged layers (3: the
// layer two ahead is fetched during a whole layer; 2: during the second
// phase only, less shared memory).  SWZ: swizzled slot layout (slot_pos).
// UT: the interface-task loop unrolled (more independent work per thread,
// more registers).  RC: the layer copied row by row (pays where a row is
// many copies per thread).  PFN: the neighbour columns' elements of the next
// layer prefetched into L2.  RPAD: floats of padding after every element row
// of a slot, so that the rows of one x-interface task batch fall into
// different banks (where a row is a multiple of 32 floats).
template <int N, int V>
struct LineShape;
struct LineDefaults {
    static constexpr bool SWZ = false, UT = false, RC = false, PFN = false;
    static constexpr int NS = 3, RPAD = 0;
    // resident CTAs per SM the batched kernel must allow (its registers then
    // match the single-mesh kernel's; 0: no bound)
    static constexpr int BMINB = 0;
};
template <> struct LineShape<1, 0> : LineDefaults { static constexpr int TX = 16, TY = 16, NS = 2, RPAD = 1; };
template <> struct LineShape<2, 0> : LineDefaults { static constexpr int TX = 8, TY = 8, NS = 2, RPAD = 8, BMINB = 2; };
template <> struct LineShape<3, 0> : LineDefaults { static constexpr int TX = 4, TY = 4, NS = 2, BMINB = 3; };
template <> struct LineShape<4, 0> : LineDefaults {
    static constexpr int TX = 2, TY = 2, NS = 2;
    static constexpr bool SWZ = true, UT = true, PFN = true;
};
template <> struct LineShape<5, 0> : LineDefaults { static constexpr int TX = 3, TY = 2, NS = 2; };
template <> struct LineShape<6, 0> : LineDefaults {
    static constexpr int TX = 3, TY = 1;
    static constexpr bool UT = true, RC = true;
};
template <> struct LineShape<7, 0> : LineDefaults {
    static constexpr int TX = 2, TY = 1;
    static constexpr bool RC = true;
};

template <int N, int TX, int TY, int NS = 3, int RPAD = 0>
struct LineTile {
    using CT = ColTile<N, TX, TY>;  // element layout in a slot, prefetch units
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int EPB = TX * TY;
    static constexpr int THREADS = ((EPB * N2 + 31) / 32) * 32;
    // fluxes [x, y][NF][N3] as node lines; element stride = N^2 (mod 32), so
    // that the N^2 threads of consecutive elements store to consecutive banks
    static constexpr int FSTR = 2 * NF * N3 + ((N2 - (2 * NF * N3) % 32) % 32 + 32) % 32;
    // x, y face fluxes [2][NF][N2][(-,+)]; element stride = 2N (mod 32)
    // (even), so that the N (-,+) pairs each element reads at a time fall into
    // consecutive banks for consecutive elements (N = 4: the column layout's)
    static constexpr int HSTR =
        N == 4 ? CT::HSTR : 4 * NF * N2 + ((2 * N - (4 * NF * N2) % 32) % 32 + 32) % 32;
    static constexpr int FREG = (EPB * FSTR + 3) / 4 * 4;  // regions in 16-byte multiples
    static constexpr int HREG = (EPB * HSTR + 3) / 4 * 4;
    // a slot: [NF][TY] element rows of TX elements (ESTR apart), RSTR apart
    static constexpr int RSTR = TX * CT::ESTR + RPAD;
    static constexpr int QSLOT = (NF * TY * RSTR + 3) / 4 * 4;
    static constexpr size_t FLOATS = (size_t)NS * QSLOT + (size_t)FREG + (size_t)HREG + CT::OPSF;
    // offset of field n of slot element el (= b * TX + a)
    __device__ static constexpr int eoff(int n, int el)
    {
        if constexpr (RPAD == 0) return (n * EPB + el) * CT::ESTR;
        else return (n * TY + el / TX) * RSTR + (el % TX) * CT::ESTR;
    }
    static constexpr size_t BYTES = FLOATS * sizeof(float);
    static constexpr int XT = (TX + 1) * TY * N2, YT = (TY + 1) * TX * N2;
};

// trace of a staged node line (element el of the slot) at one end; base is
// the line's first node (line_base)
template <class LT, int N, int DIR, bool SWZ>
__device__ __forceinline__ void slot_trace(const float *slot, int el, int base, const float *l,
                                           float q[NF])
{
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? N : N * N);
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        const float *e = slot + LT::eoff(n, el);
        float v[N];
        if constexpr (DIR == 0) {
            load_line<N>(e + slot_pos<N, SWZ>(base), v);   // an x line is one 16-byte unit
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = e[slot_pos<N, SWZ>(base + c * stride)];
        }
        q[n] = line_dot<N>(l, v);
    }
}

// x (DIR 0) or y (DIR 1) interface a in [0, len] of row r at face point pt,
// both traces from node lines (staged, or the neighbour column's in DRAM/L2)
template <class LT, int N, int TX, int TY, int DIR, typename Ix, bool SWZ>
__device__ __forceinline__ void slot_interface(const float *__restrict__ Qin, const float *slot,
                                               float *sH, const Geo &g, const float *lm,
                                               const float *lp, float gamma, float gm1, int a,
                                               int r, int len, Ix e_lo, Ix e_hi, int pt)
{
    constexpr int N2 = LT::N2;
    const int base = line_base<N, DIR>(pt % N, pt / N);
    auto local = [&](int c) { return DIR == 0 ? r * TX + c : c * TX + r; };
    float qL[NF], qR[NF];
    if (a == 0) global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_lo, base, lp, qL);
    else slot_trace<LT, N, DIR, SWZ>(slot, local(a - 1), base, lp, qL);
    if (a == len) global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_hi, base, lm, qR);
    else slot_trace<LT, N, DIR, SWZ>(slot, local(a), base, lm, qR);
    float f[NF];
    lf_flux2_f<DIR>(qL, qR, gamma, gm1, f);
    if (a > 0) {
        float *h = sH + (size_t)local(a - 1) * LT::HSTR + (DIR * NF * N2 + pt) * 2 + 1;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
    if (a < len) {
        float *h = sH + (size_t)local(a) * LT::HSTR + (DIR * NF * N2 + pt) * 2 + 0;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
}

// One column chunk of the stage, block = column + chunk x columns of the mesh
// (the CTA's index in a launch over one mesh); MODE and Ix as for
// column_stage_kernel.  Run by exactly LineTile::THREADS threads: the copy
// offsets and the interface-task loop stride assume that block size.
template <int N, int V, int MODE, typename Ix>
__device__ __forceinline__ void line_stage_body(const float *__restrict__ Qin,
                                                float *__restrict__ Out, float *__restrict__ dQ,
                                                const Ops<float> &T, const Geo &g, float A,
                                                float B, const double *__restrict__ dt, int zchunk,
                                                unsigned block)
{
    constexpr int TX = LineShape<N, V>::TX, TY = LineShape<N, V>::TY;
    constexpr bool SWZ = LineShape<N, V>::SWZ;
    constexpr int NS = LineShape<N, V>::NS;
    static_assert(NS == 2 || NS == 3, "two or three staging slots");
    using LT = LineTile<N, TX, TY, NS, LineShape<N, V>::RPAD>;
    using CT = ColTile<N, TX, TY>;
    constexpr int N2 = LT::N2, N3 = LT::N3, EPB = LT::EPB;
    constexpr int FSTR = LT::FSTR, HSTR = LT::HSTR, ESTR = CT::ESTR;
    extern __shared__ __align__(16) float lsm[];
    float *slots = lsm;                            // [NS][QSLOT]
    float *sF = slots + NS * LT::QSLOT;            // [EPB][FSTR]
    float *sH = sF + LT::FREG;                     // [EPB][HSTR]
    float *sOp = sH + LT::HREG;                    // D[3][N][N], Lm[3][N], Lp[3][N], lm[N], lp[N]

    const int ncx = (g.nx + TX - 1) / TX, ncy = (g.ny + TY - 1) / TY;
    const int col = (int)(block % (unsigned)(ncx * ncy));
    const int chunk = (int)(block / (unsigned)(ncx * ncy));
    const int ex0 = (col % ncx) * TX, ey0 = (col / ncx) * TY;
    const int txv = min(TX, g.nx - ex0), tyv = min(TY, g.ny - ey0);
    const int z0 = chunk * zchunk;
    const int z1 = min(g.nz, z0 + zchunk);
    const float dtr = MODE != 0 ? (float)(*dt) : 0.0f;
    const float gamma = T.gamma, gm1 = T.gm1;

    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int t = tid; t < 3 * N2 + 6 * N; t += nthr) {
        float v;
        if (t < 3 * N2) v = T.D[t / N2][(t % N2) / N][t % N];
        else if (t < 3 * N2 + 3 * N) v = T.Lm[(t - 3 * N2) / N][(t - 3 * N2) % N];
        else v = T.Lp[(t - 3 * N2 - 3 * N) / N][(t - 3 * N2 - 3 * N) % N];
        sOp[t] = v;
    }
    for (int t = tid; t < 2 * N; t += nthr) sOp[3 * N2 + 6 * N + t] = t < N ? T.lm[t] : T.lp[t - N];
    const float *lm = sOp + 3 * N2 + 6 * N, *lp = lm + N;

    const int exL = (ex0 - 1 + g.nx) % g.nx, exR = (ex0 + txv) % g.nx;
    const int eyL = (ey0 - 1 + g.ny) % g.ny, eyR = (ey0 + tyv) % g.ny;
    const Ix plane = (Ix)g.nx * g.ny;
    const Ix E = (Ix)g.E;

    // this thread's z line (i, j) of element el
    const int el = tid / N2;
    const int ln = tid - el * N2;
    const int a = el % TX, b = el / TX;
    const bool active = el < EPB && a < txv && b < tyv;
    const int i = ln % N, j = ln / N;

    auto slot_of = [&](int L) { return slots + ((L - z0 + 1) % NS) * LT::QSLOT; };
    auto zmod = [&](int L) { return (L % g.nz + g.nz) % g.nz; };
    // node line (i, j) of this thread's element in a slot, per field
    auto load_zline = [&](const float *slot, float v[NF][N]) {
#pragma unroll
        for (int n = 0; n < NF; ++n)
#pragma unroll
            for (int c = 0; c < N; ++c)
                v[n][c] = slot[LT::eoff(n, el) + slot_pos<N, SWZ>((c * N + j) * N + i)];
    };
    // This thread's share of a layer's copy: the same units every layer, so
    // their offsets (source relative to the layer, destination relative to
    // the slot) are computed once (W = 4: 16-byte units; else per layer).
    constexpr int W = CT::W, RU = CT::ROW_UNITS;
    constexpr int UNITS = NF * TY * RU;
    constexpr int MAXC = (UNITS + LT::THREADS - 1) / LT::THREADS;
    constexpr bool PRE = W == 4 && MAXC <= 6;
    Ix csrc[PRE ? MAXC : 1];
    int cdst[PRE ? MAXC : 1];
    if constexpr (PRE) {
#pragma unroll
        for (int m = 0; m < MAXC; ++m) {
            const int t = tid + m * LT::THREADS;
            const int n = t / (TY * RU);
            const int r = t - n * (TY * RU);
            const int bb = r / RU;
            const int u = r - bb * RU;
            cdst[m] = -1;
            csrc[m] = 0;
            if (t < UNITS && bb < tyv && u * W < txv * N3) {
                const int ea = (u * W) / N3, o = u * W - ea * N3;
                csrc[m] = ((Ix)n * E + ex0 + (Ix)g.nx * (ey0 + bb)) * N3 + u * W;
                cdst[m] = LT::eoff(n, bb * TX + ea) + slot_pos<N, SWZ>(o);
            }
        }
    }
    auto prefetch = [&](int L) {
        if constexpr (PRE) {
            const float *src = Qin + plane * (Ix)zmod(L) * N3;
            float *dst = slot_of(L);
#pragma unroll
            for (int m = 0; m < MAXC; ++m)
                if (cdst[m] >= 0) cp_async16(dst + cdst[m], src + csrc[m]);
            cp_async_commit();
        } else if constexpr (LineShape<N, V>::RC) {
            static_assert(ESTR == N3 && !SWZ, "row copies need unpadded, unswizzled slots");
            // unpadded slots: each (field, element row) of the layer is one
            // contiguous run in DRAM and in the slot, copied unit by unit
            const Ix lay = plane * (Ix)zmod(L);
            float *dst0 = slot_of(L);
            const int len = txv * N3 / W;
#pragma unroll 1
            for (int row = 0; row < NF * TY; ++row) {
                const int n = row / TY, bb = row - n * TY;
                if (bb >= tyv) continue;
                const float *src = Qin + ((Ix)n * E + ex0 + (Ix)g.nx * (ey0 + bb) + lay) * N3;
                float *dst = dst0 + LT::eoff(n, bb * TX);
                for (int u = tid; u < len; u += LT::THREADS) {
                    if constexpr (W == 4) cp_async16(dst + 4 * u, src + 4 * u);
                    else cp_async4(dst + u, src + u);
                }
            }
            cp_async_commit();
        } else if constexpr (LineShape<N, V>::RPAD == 0) {
            column_prefetch<N, TX, TY, Ix, SWZ>(Qin, slot_of(L), g, ex0, ey0, txv, tyv, zmod(L));
        } else {
            // the column kernel's unit loop, into the padded rows
            const Ix lay = plane * (Ix)zmod(L);
            float *dst0 = slot_of(L);
            for (int t = tid; t < UNITS; t += LT::THREADS) {
                const int n = t / (TY * RU);
                const int r = t - n * (TY * RU);
                const int bb = r / RU;
                const int u = r - bb * RU;
                if (bb >= tyv || u * W >= txv * N3) continue;
                const int ea = (u * W) / N3, o = u * W - ea * N3;
                const float *src = Qin + ((Ix)n * E + ex0 + (Ix)g.nx * (ey0 + bb) + lay) * N3 + u * W;
                float *dst = dst0 + LT::eoff(n, bb * TX + ea) + slot_pos<N, SWZ>(o);
                if constexpr (W == 4) cp_async16(dst, src);
                else cp_async4(dst, src);
            }
            cp_async_commit();
        }
    };

    prefetch(z0 - 1);
    prefetch(z0);
    if constexpr (NS == 3) prefetch(z0 + 1);
    cp_async_wait_all();
    __syncthreads();

    // operator values of this thread's line, for the whole chunk
    float lmr[N], lpr[N], dx[N], dy[N];
    load_line<N>(lm, lmr);
    load_line<N>(lp, lpr);
    load_line<N>(sOp + 0 * N2 + i * N, dx);
    load_line<N>(sOp + 1 * N2 + j * N, dy);
    const float *Lm = sOp + 3 * N2, *Lp = Lm + 3 * N;
    const float lmx = Lm[i], lmy = Lm[N + j], lpx = Lp[i], lpy = Lp[N + j];

    // z slabs: this line's face point in the halo layout [NF][nx*ny][N^2]
    const Ix hcol = ((Ix)(ex0 + a) + (Ix)g.nx * (ey0 + b)) * N2 + j * N + i;
    const Ix hstride = plane * N2;

    // flux through the -z face of the line in the current layer (a slab's
    // first layer: the layer below is another slab's, known by its traces)
    float fzm[NF];
    if (active) {
        float v[NF][N], tp[NF], tm[NF];
        if (g.zlo != nullptr && z0 == 0) {
#pragma unroll
            for (int n = 0; n < NF; ++n) tp[n] = static_cast<const float *>(g.zlo)[hcol + n * hstride];
        } else {
            load_zline(slot_of(z0 - 1), v);
#pragma unroll
            for (int n = 0; n < NF; ++n) tp[n] = line_dot<N>(lpr, v[n]);
        }
        load_zline(slot_of(z0), v);
#pragma unroll
        for (int n = 0; n < NF; ++n) tm[n] = line_dot<N>(lmr, v[n]);
        lf_flux2_f<2>(tp, tm, gamma, gm1, fzm);
    }
    __syncthreads();
    if constexpr (NS == 3) {
        if (z0 + 2 <= z1) prefetch(z0 + 2);
    } else {
        prefetch(z0 + 1);   // into the slot of z0 - 1, free now
        cp_async_wait_all();
        __syncthreads();
    }

    for (int z = z0; z < z1; ++z) {
        const float *cur = slot_of(z), *nxt = slot_of(z + 1);
        const Ix e = ex0 + a + (Ix)g.nx * (ey0 + b) + plane * z;

        // the neighbour columns' elements of the next layer into L2 (PFN):
        // their node lines are the interface tasks' only reads from DRAM
        if constexpr (LineShape<N, V>::PFN) {
            constexpr int LPE = (N3 * 4 + 127) / 128 + 1;  // cache lines an element spans
            if (z + 1 < z1) {
                const Ix zn = plane * (Ix)(z + 1);
                for (int t = tid; t < NF * 2 * (TX + TY) * LPE; t += LT::THREADS) {
                    const int n = t / (2 * (TX + TY) * LPE), r = t - n * (2 * (TX + TY) * LPE);
                    const int k = r / LPE, l = r - k * LPE;
                    Ix e2;
                    if (k < 2 * TY) {  // left / right neighbour column's row
                        const int row = k >> 1;
                        if (row >= tyv) continue;
                        e2 = (k & 1 ? exR : exL) + (Ix)g.nx * (ey0 + row) + zn;
                    } else {           // front / back
                        const int cx = (k - 2 * TY) >> 1;
                        if (cx >= txv) continue;
                        e2 = ex0 + cx + (Ix)g.nx * (k & 1 ? eyR : eyL) + zn;
                    }
                    const char *a = reinterpret_cast<const char *>(Qin + ((Ix)n * E + e2) * N3);
                    const char *q = a + 128 * l;
                    if (q < a + N3 * sizeof(float)) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
                }
            }
        }

        // P: node fluxes, the z interface above the line, x and y interfaces
        float qc[NF][N], fz[NF][N], fzp[NF], dq[NF][N];
        if (active) {
            if (MODE != 0 && A != 0.0f) {
#pragma unroll
                for (int n = 0; n < NF; ++n)
#pragma unroll
                    for (int c = 0; c < N; ++c)
                        dq[n][c] = dQ[((Ix)n * E + e) * N3 + (c * N + j) * N + i];
            }
            load_zline(cur, qc);
            float *sx = sF + (size_t)el * FSTR;
            float *sy = sx + NF * N3;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                float q[NF], fx[NF], fy[NF], f3[NF];
#pragma unroll
                for (int n = 0; n < NF; ++n) q[n] = qc[n][c];
                node_flux_f(q, gm1, fx, fy, f3);
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    sx[n * N3 + (c * N + j) * N + i] = fx[n];
                    sy[n * N3 + (c * N + i) * N + j] = fy[n];
                    fz[n][c] = f3[n];
                }
            }
            float v[NF][N], tp[NF], tm[NF];
            if (g.zhi != nullptr && z == g.nz - 1) {
                // a slab's last layer: the layer above is another slab's
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    tp[n] = line_dot<N>(lpr, qc[n]);
                    tm[n] = static_cast<const float *>(g.zhi)[hcol + n * hstride];
                }
            } else {
                load_zline(nxt, v);
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    tp[n] = line_dot<N>(lpr, qc[n]);
                    tm[n] = line_dot<N>(lmr, v[n]);
                }
            }
            lf_flux2_f<2>(tp, tm, gamma, gm1, fzp);
        }
        // interface task t: the local Lax-Friedrichs flux at one x or y face point
        auto task = [&](int t) {
            if (t < LT::XT) {
                // interface index slowest, so that a warp shares its source
                const int ai = t / (TY * N2), r = t - ai * (TY * N2);
                const int row = r / N2, pt = r - row * N2;
                if (ai > txv || row >= tyv) return;
                const Ix er = (Ix)g.nx * (ey0 + row) + plane * z;
                slot_interface<LT, N, TX, TY, 0, Ix, SWZ>(Qin, cur, sH, g, lm, lp, gamma, gm1, ai, row,
                                                 txv, exL + er, exR + er, pt);
            } else {
                const int u = t - LT::XT;
                const int ai = u / (TX * N2), r = u - ai * (TX * N2);
                const int cx = r / N2, pt = r - cx * N2;
                if (ai > tyv || cx >= txv) return;
                const Ix ec = ex0 + cx + plane * z;
                slot_interface<LT, N, TX, TY, 1, Ix, SWZ>(Qin, cur, sH, g, lm, lp, gamma, gm1, ai, cx,
                                                 tyv, ec + (Ix)g.nx * eyL, ec + (Ix)g.nx * eyR, pt);
            }
        };
        if constexpr (LineShape<N, V>::UT) {
#pragma unroll
            for (int t = tid; t < LT::XT + LT::YT; t += LT::THREADS) task(t);
        } else {
            for (int t = tid; t < LT::XT + LT::YT; t += LT::THREADS) task(t);
        }
        __syncthreads();
        // two slots: the slot of layer z is free once every thread is past P
        if constexpr (NS == 2)
            if (z + 2 <= z1) prefetch(z + 2);

        // G: derivative, lift, update of the line's nodes
        if (active) {
            const float *h = sH + (size_t)el * HSTR;
            const float *fxl = sF + (size_t)el * FSTR;
            const float *fyl = fxl + NF * N3;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                float dz[N];
                load_line<N>(sOp + 2 * N2 + c * N, dz);
                const float lmz = Lm[2 * N + c], lpz = Lp[2 * N + c];
                const int node = (c * N + j) * N + i, px = c * N + j, py = c * N + i;
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    float vx[N], vy[N];
                    load_line<N>(fxl + n * N3 + px * N, vx);
                    load_line<N>(fyl + n * N3 + py * N, vy);
                    float2 a2 = f2(0.0f, 0.0f);
                    a2 = dot2_acc<N>(dx, vx, a2);
                    a2 = dot2_acc<N>(dy, vy, a2);
                    a2 = dot2_acc<N>(dz, fz[n], a2);
                    const float2 hx = *reinterpret_cast<const float2 *>(h + ((0 * NF + n) * N2 + px) * 2);
                    const float2 hy = *reinterpret_cast<const float2 *>(h + ((1 * NF + n) * N2 + py) * 2);
                    a2 = __ffma2_rn(f2(lmx, -lpx), hx, a2);
                    a2 = __ffma2_rn(f2(lmy, -lpy), hy, a2);
                    a2 = __ffma2_rn(f2(lmz, -lpz), f2(fzm[n], fzp[n]), a2);
                    const float acc = __fadd_rn(a2.x, a2.y);
                    const Ix o = ((Ix)n * E + e) * N3 + node;
                    if (MODE == 0) {
                        Out[o] = acc;
                    } else {
                        const float d = __fmaf_rn(dtr, acc, A == 0.0f ? 0.0f : __fmul_rn(A, dq[n][c]));
                        dQ[o] = d;
                        if (MODE == 1) Out[o] = __fmaf_rn(B, d, qc[n][c]);
                    }
                }
            }
#pragma unroll
            for (int n = 0; n < NF; ++n) fzm[n] = fzp[n];
        }
        // the fluxes, face fluxes and (three slots) the slot of layer z are
        // free once every thread is past G
        cp_async_wait_all();
        __syncthreads();
        if constexpr (NS == 3)
            if (z + 3 <= z1) prefetch(z + 3);
    }
}

// The stage over one mesh: one CTA per (column, z chunk).
template <int N, int V, int MODE, typename Ix>
__global__ void __launch_bounds__(
    LineTile<N, LineShape<N, V>::TX, LineShape<N, V>::TY, LineShape<N, V>::NS,
             LineShape<N, V>::RPAD>::THREADS)
    line_stage_kernel(const float *__restrict__ Qin, float *__restrict__ Out,
                      float *__restrict__ dQ, const Ops<float> T, const Geo g, float A, float B,
                      const double *__restrict__ dt, int zchunk)
{
    line_stage_body<N, V, MODE, Ix>(Qin, Out, dQ, T, g, A, B, dt, zchunk, blockIdx.x);
}

// The stage over the instances of one degree of a batch: one CTA per work
// item (instance, column, z chunk), the same body as line_stage_kernel, so
// an instance's floats are those of the same mesh stepped alone.  parity 0:
// the stage reads Q and writes the second state Qt; 1: the reverse.
template <int N, int MODE, typename Ix>
__global__ void __launch_bounds__(
    LineTile<N, LineShape<N, 0>::TX, LineShape<N, 0>::TY, LineShape<N, 0>::NS,
             LineShape<N, 0>::RPAD>::THREADS, LineShape<N, 0>::BMINB)
    batched_line_kernel(const LineItem *__restrict__ items, const InstDev *__restrict__ inst,
                        int parity, float A, float B)
{
    // the instance's geometry staged in shared memory: the body reads it
    // where the single-mesh kernel reads its parameter bank, without holding
    // it in registers
    __shared__ Geo sg;
    const LineItem it = items[blockIdx.x];
    const InstDev *I = inst + it.inst;
    if (threadIdx.x == 0) sg = I->g;
    __syncthreads();
    line_stage_body<N, 0, MODE, Ix>(parity ? I->Qt : I->Q, parity ? I->Q : I->Qt, I->dQ, I->T, sg,
                                    A, B, I->dt, it.zchunk, (unsigned)it.block);
}
