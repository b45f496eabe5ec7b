// dg_column.cuh -- the float form's single-mesh RK stage as a z-marching
// column kernel.  Included by dg_kernels.cuh (inside namespace dg).
//
// A CTA owns a column of TX x TY elements in x-y and walks it layer by layer
// in z over a chunk of layers.  The state of the layers ahead is prefetched
// into a ring of three shared-memory slots with cp.async while the current
// layer computes, so DRAM latency overlaps the arithmetic.  Per layer:
//
//   B  every thread: the Euler fluxes of its node (Eq. 2-3) -> shared memory;
//      line tasks: the traces of each element's face-normal node lines at
//      the line's ends (x and y lines both ends, z lines of this layer the +z
//      end, z lines of the next layer the -z end) -> shared memory
//   D  interface tasks: the local Lax-Friedrichs flux (Sec. II.B) at every
//      face point of the column's layer, each interface once: x and y
//      interfaces inside the column from the traces of both sides, at the
//      column's boundary with the neighbour column's trace interpolated from
//      its node line (read through L2); the z interface to the next layer
//      from this layer's +z and the next layer's -z traces, kept for the next
//      layer as its -z face flux
//   G  every thread: sum-factorised weak derivative, lift of the six face
//      fluxes, and the stage update of its node -> DRAM
//
// A boundary interface is evaluated by both columns that share it, from
// bitwise-identical traces (one function, one operation order, for the
// shared-memory and the global source) in the same argument order, so both
// see the same flux and discrete conservation holds.  Output goes to a second
// state buffer, because neighbouring columns still read the input state.
#pragma once

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Column cross-sections per N (= p + 1): about 256 nodes per layer.
template <int N, int V>
struct ColShape;
template <> struct ColShape<1, 0> { static constexpr int TX = 8, TY = 8; };
template <> struct ColShape<2, 0> { static constexpr int TX = 8, TY = 4; };
template <> struct ColShape<3, 0> { static constexpr int TX = 3, TY = 3; };
template <> struct ColShape<4, 0> { static constexpr int TX = 2, TY = 2; };
template <> struct ColShape<5, 0> { static constexpr int TX = 2, TY = 1; };
template <> struct ColShape<6, 0> { static constexpr int TX = 1, TY = 1; };
template <> struct ColShape<7, 0> { static constexpr int TX = 1, TY = 1; };

template <int N, int TX, int TY>
struct ColTile {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int EPB = TX * TY;
    static constexpr int THREADS = ((EPB * N3 + 31) / 32) * 32;
    static constexpr int pad16(int x) { return x + ((16 - x % 32) + 32) % 32; }
    // one layer's state [NF][EPB][ESTR] (element rows in DRAM order); 16-byte
    // aligned slots
    // element stride inside a slot: N^3 padded by 16 floats when N^3 is a
    // multiple of 32, so that two elements' nodes fall into different bank
    // halves (the strided y/z node-line loads of neighbouring elements would
    // otherwise collide); the per-thread cp.async places each unit anyway
    static constexpr int ESTR = N3 % 32 == 0 ? N3 + 16 : N3;
    static constexpr int QSLOT = ((NF * EPB * ESTR + 3) / 4) * 4;
    static constexpr int FSTR = pad16(3 * NF * N3);      // fluxes [3][NF][N3], direction-major
    static constexpr int TSTR = pad16(6 * NF * N2);      // traces [face = 2 dir + side][NF][N2]
    static constexpr int HSTR = pad16(2 * NF * N2 * 2);  // x, y face fluxes [2][NF][N2][(-,+)]
    static constexpr int ZSTR = NF * N2;                 // z face fluxes [NF][N2]
    static constexpr int OPSF = ((3 * N2 + 8 * N + 3) / 4) * 4;  // D, Lm, Lp, lm, lp
    static constexpr size_t FLOATS =
        (size_t)3 * QSLOT + (size_t)EPB * (FSTR + TSTR + HSTR) + 2 * EPB * ZSTR + OPSF;
    static constexpr size_t BYTES = FLOATS * sizeof(float);
    // unit of the prefetch: 16 bytes where every element row starts 16-byte
    // aligned (N^3 a multiple of 4), else one float
    static constexpr int W = N3 % 4 == 0 ? 4 : 1;
    static constexpr int ROW_UNITS = TX * N3 / W;
    // tasks of the two task phases per layer
    static constexpr int LINE_TASKS = 4 * EPB * N2;
    static constexpr int XT = (TX + 1) * TY * N2, YT = (TY + 1) * TX * N2, ZT = EPB * N2;
};

// Packed float pairs: one FFMA2 / FMUL2 / FADD2 instruction does two
// independent IEEE operations (sm_100 and later), so paired work issues half
// the floating-point instructions with the same rounding per lane.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Trace sum_c l[c] v(c) of a node line, with the same explicitly ordered
// operations for every source (shared or global memory), so that two columns
// computing the same trace get the same float: even and odd nodes summed in
// the two lanes of a packed pair, then added.
template <int N>
__device__ __forceinline__ float line_dot(const float *l, const float v[N])
{
    if constexpr (N == 1) {
        return __fmul_rn(l[0], v[0]);
    } else {
        float2 s = __fmul2_rn(f2(l[0], l[1]), f2(v[0], v[1]));
#pragma unroll
        for (int c = 2; c + 1 < N; c += 2) s = __ffma2_rn(f2(l[c], l[c + 1]), f2(v[c], v[c + 1]), s);
        if constexpr (N % 2 == 1) s.x = __fmaf_rn(l[N - 1], v[N - 1], s.x);
        return __fadd_rn(s.x, s.y);
    }
}

// acc + sum_c d[c] v[c] into a packed accumulator (even c in .x, odd in .y)
template <int N>
__device__ __forceinline__ float2 dot2_acc(const float d[N], const float v[N], float2 acc)
{
#pragma unroll
    for (int c = 0; c + 1 < N; c += 2) acc = __ffma2_rn(f2(d[c], d[c + 1]), f2(v[c], v[c + 1]), acc);
    if constexpr (N % 2 == 1) acc.x = __fmaf_rn(d[N - 1], v[N - 1], acc.x);
    return acc;
}

template <int N, int DIR>
__device__ __forceinline__ void line_values(const float *p, float v[N])
{
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? N : N * N);
    if constexpr (DIR == 0) {
        load_line<N>(p, v);
    } else {
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] = p[c * stride];
    }
}

// first node of the face-normal line through face point (t1, t2)
template <int N, int DIR>
__device__ __forceinline__ int line_base(int t1, int t2)
{
    return DIR == 0 ? (t2 * N + t1) * N : (DIR == 1 ? t2 * N * N + t1 : t2 * N + t1);
}

// trace of an element of the neighbour column, from DRAM/L2 (Ix: the index
// type of the mesh's arrays, 32-bit when every offset fits)
template <int N, int DIR, typename Ix>
__device__ __forceinline__ void global_trace(const float *__restrict__ Q, Ix E, Ix e, int base,
                                             const float *l, float q[NF])
{
    constexpr int N3 = N * N * N;
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        float v[N];
        line_values<N, DIR>(Q + ((Ix)n * E + e) * N3 + base, v);
        q[n] = line_dot<N>(l, v);
    }
}

// 2 F* of the local Lax-Friedrichs flux through a face with normal +e_DIR:
// the two sides' pressure, normal velocity, flux and speed evaluated as
// packed pairs (left in .x, right in .y), every operation explicitly rounded.
template <int DIR>
__device__ __forceinline__ void lf_flux2_f(const float qL[NF], const float qR[NF], float gamma,
                                           float gm1, float f[NF])
{
    float2 q[NF];
#pragma unroll
    for (int n = 0; n < NF; ++n) q[n] = f2(qL[n], qR[n]);
    const float2 rinv = f2(fast_rcp(qL[0]), fast_rcp(qR[0]));
    float2 mm = __fmul2_rn(q[1], q[1]);
    mm = __ffma2_rn(q[2], q[2], mm);
    mm = __ffma2_rn(q[3], q[3], mm);
    // p = (gamma - 1) (E - |m|^2 / (2 rho))
    const float2 p = __fmul2_rn(f2(gm1, gm1), __ffma2_rn(f2(-0.5f, -0.5f), __fmul2_rn(mm, rinv), q[4]));
    const float2 un = __fmul2_rn(q[1 + DIR], rinv);
    const float2 c2 = __fmul2_rn(__fmul2_rn(f2(gamma, gamma), p), rinv);
    const float lam = fmaxf(__fadd_rn(fabsf(un.x), fast_sqrt(c2.x)),
                            __fadd_rn(fabsf(un.y), fast_sqrt(c2.y)));
    float2 F[NF];
    F[0] = q[1 + DIR];
#pragma unroll
    for (int n = 1; n < 4; ++n) F[n] = n == DIR + 1 ? __ffma2_rn(q[n], un, p) : __fmul2_rn(q[n], un);
    F[4] = __fmul2_rn(__fadd2_rn(q[4], p), un);
#pragma unroll
    for (int n = 0; n < NF; ++n)
        f[n] = __fmaf_rn(-lam, __fsub_rn(qR[n], qL[n]), __fadd_rn(F[n].x, F[n].y));
}

// Euler fluxes of one node (Eq. 2-3) in the three directions, every
// operation explicitly rounded so that the column kernels agree bitwise.
__device__ __forceinline__ void node_flux_f(const float q[NF], float gm1, float fx[NF],
                                            float fy[NF], float fz[NF])
{
    const float rinv = fast_rcp(q[0]);
    const float u = __fmul_rn(q[1], rinv), v = __fmul_rn(q[2], rinv), w = __fmul_rn(q[3], rinv);
    const float m2 = __fmaf_rn(q[3], w, __fmaf_rn(q[2], v, __fmul_rn(q[1], u)));
    const float p = __fmul_rn(gm1, __fmaf_rn(-0.5f, m2, q[4]));
    const float ep = __fadd_rn(q[4], p);
    fx[0] = q[1];
    fx[1] = __fmaf_rn(q[1], u, p);
    fx[2] = __fmul_rn(q[2], u);
    fx[3] = __fmul_rn(q[3], u);
    fx[4] = __fmul_rn(ep, u);
    fy[0] = q[2];
    fy[1] = __fmul_rn(q[1], v);
    fy[2] = __fmaf_rn(q[2], v, p);
    fy[3] = __fmul_rn(q[3], v);
    fy[4] = __fmul_rn(ep, v);
    fz[0] = q[3];
    fz[1] = __fmul_rn(q[1], w);
    fz[2] = __fmul_rn(q[2], w);
    fz[3] = __fmaf_rn(q[3], w, p);
    fz[4] = __fmul_rn(ep, w);
}

// Position in a slot of the node at offset o = (k N + j) N + i of its
// element.  SWZ (N = 4 only): the 16-byte x-line (j, k) is stored at line
// 4 k + (j xor r(k)), r(k) the bit reversal of k, so that both the z lines
// (fixed i, j) and the y lines (fixed i, k) of two neighbouring elements
// read by one warp fall into 32 distinct banks.
template <int N, bool SWZ>
__device__ __forceinline__ int slot_pos(int o)
{
    if constexpr (SWZ) {
        static_assert(N == 4, "the slot swizzle is defined for N = 4");
        const int k = o >> 4, j = (o >> 2) & 3;
        return ((k << 2) | (j ^ (((k & 1) << 1) | (k >> 1)))) * 4 + (o & 3);
    } else {
        return o;
    }
}

// Copy layer zl (periodic) of the column into a slot: whole valid rows.
template <int N, int TX, int TY, typename Ix, bool SWZ = false>
__device__ __forceinline__ void column_prefetch(const float *__restrict__ Q, float *slot,
                                                const Geo &g, int ex0, int ey0, int txv, int tyv,
                                                int zl)
{
    using CT = ColTile<N, TX, TY>;
    constexpr int N3 = CT::N3, W = CT::W, RU = CT::ROW_UNITS, EPB = CT::EPB;
    const Ix plane = (Ix)g.nx * g.ny;
    for (int t = threadIdx.x; t < NF * TY * RU; t += blockDim.x) {
        const int n = t / (TY * RU);
        const int r = t - n * (TY * RU);
        const int b = r / RU;
        const int u = r - b * RU;
        if (b >= tyv || u * W >= txv * N3) continue;
        const Ix e0 = ex0 + (Ix)g.nx * (ey0 + b) + plane * zl;
        const float *src = Q + ((Ix)n * (Ix)g.E + e0) * N3 + u * W;
        const int a = (u * W) / N3, o = u * W - a * N3;  // element of the row, node offset
        float *dst = slot + (n * EPB + b * TX + a) * CT::ESTR + slot_pos<N, SWZ>(o);
        if constexpr (W == 4) cp_async16(dst, src);
        else cp_async4(dst, src);
    }
    cp_async_commit();
}

// Line tasks of layer z (traces of this layer's x and y lines, both ends, and
// of its z lines, + end) and of the next layer (z lines, - end).
template <int N, int TX, int TY, int DIR>
__device__ __forceinline__ void line_task(const float *slot, float *sT, const float *lm,
                                          const float *lp, int el, int ln, int which)
{
    using CT = ColTile<N, TX, TY>;
    constexpr int N2 = CT::N2, EPB = CT::EPB;
    const int t1 = ln % N, t2 = ln / N;
    const int base = line_base<N, DIR>(t1, t2);
    float *t = sT + (size_t)el * CT::TSTR;
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        float v[N];
        line_values<N, DIR>(slot + (n * EPB + el) * CT::ESTR + base, v);
        if (which != 1) t[((2 * DIR + 0) * NF + n) * N2 + ln] = line_dot<N>(lm, v);
        if (which != 0) t[((2 * DIR + 1) * NF + n) * N2 + ln] = line_dot<N>(lp, v);
    }
}

// x (DIR 0) or y (DIR 1) interface task: interface a in [0, len] along DIR of
// row r (the other in-plane index); a = 0 and a = len are the column's
// boundaries, whose outer trace comes from the neighbour column.
template <int N, int TX, int TY, int DIR, typename Ix>
__device__ __forceinline__ void plane_interface(const float *__restrict__ Qin, const float *sT,
                                                float *sH, const Geo &g, const float *lm,
                                                const float *lp, float gamma, float gm1, int a,
                                                int r, int len, Ix e_lo, Ix e_hi, int pt)
{
    using CT = ColTile<N, TX, TY>;
    constexpr int N2 = CT::N2;
    const int t1 = pt % N, t2 = pt / N;
    // in-column element at in-plane index c along DIR of this row
    auto local = [&](int c) { return DIR == 0 ? r * TX + c : c * TX + r; };
    float qL[NF], qR[NF];
    if (a == 0) {
        global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_lo, line_base<N, DIR>(t1, t2), lp, qL);
    } else {
        const float *t = sT + (size_t)local(a - 1) * CT::TSTR + (2 * DIR + 1) * NF * N2 + pt;
#pragma unroll
        for (int n = 0; n < NF; ++n) qL[n] = t[n * N2];
    }
    if (a == len) {
        global_trace<N, DIR, Ix>(Qin, (Ix)g.E, e_hi, line_base<N, DIR>(t1, t2), lm, qR);
    } else {
        const float *t = sT + (size_t)local(a) * CT::TSTR + (2 * DIR + 0) * NF * N2 + pt;
#pragma unroll
        for (int n = 0; n < NF; ++n) qR[n] = t[n * N2];
    }
    float f[NF];
    lf_flux2_f<DIR>(qL, qR, gamma, gm1, f);
    if (a > 0) {
        float *h = sH + (size_t)local(a - 1) * CT::HSTR + (DIR * NF * N2 + pt) * 2 + 1;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
    if (a < len) {
        float *h = sH + (size_t)local(a) * CT::HSTR + (DIR * NF * N2 + pt) * 2 + 0;
#pragma unroll
        for (int n = 0; n < NF; ++n) h[n * N2 * 2] = f[n];
    }
}

// One column chunk of the stage.  MODE 0 writes the rhs to Out, MODE 1 the
// LSERK stage update (dQ <- A dQ + dt R, Out <- Qin + B dQ), MODE 2 a step's
// last stage, whose dQ no later stage reads: only Out <- Qin + B (A dQ + dt R),
// dQ left as it was.  Ix is the index
// type of the state arrays: int when 5 E N^3 fits (32-bit address arithmetic
// is measurably cheaper here), else a 64-bit integer.
// (shared memory holds about four CTAs per SM; registers are sized for that)
template <int N, int V, int MODE, typename Ix>
__global__ void __launch_bounds__(ColTile<N, ColShape<N, V>::TX, ColShape<N, V>::TY>::THREADS,
                                  1024 / ColTile<N, ColShape<N, V>::TX, ColShape<N, V>::TY>::THREADS)
    column_stage_kernel(const float *__restrict__ Qin, float *__restrict__ Out,
                        float *__restrict__ dQ, const Ops<float> T, const Geo g, float A,
                        float B, const double *__restrict__ dt, int zchunk)
{
    constexpr int TX = ColShape<N, V>::TX, TY = ColShape<N, V>::TY;
    using CT = ColTile<N, TX, TY>;
    constexpr int N2 = CT::N2, N3 = CT::N3, EPB = CT::EPB;
    constexpr int FSTR = CT::FSTR, TSTR = CT::TSTR, HSTR = CT::HSTR, ZSTR = CT::ZSTR;
    extern __shared__ __align__(16) float csm[];
    float *slots = csm;                            // [3][QSLOT]
    float *sF = slots + 3 * CT::QSLOT;             // [EPB][FSTR]
    float *sT = sF + EPB * FSTR;                   // [EPB][TSTR]
    float *sH = sT + EPB * TSTR;                   // [EPB][HSTR]
    float *sZ = sH + EPB * HSTR;                   // [2][EPB][ZSTR]
    float *sOp = sZ + 2 * EPB * ZSTR;              // D[3][N][N], Lm[3][N], Lp[3][N], lm[N], lp[N]

    const int ncx = (g.nx + TX - 1) / TX, ncy = (g.ny + TY - 1) / TY;
    const int col = (int)(blockIdx.x % (unsigned)(ncx * ncy));
    const int chunk = (int)(blockIdx.x / (unsigned)(ncx * ncy));
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

    // periodic neighbour columns (element coordinates of the halo rows)
    const int exL = (ex0 - 1 + g.nx) % g.nx, exR = (ex0 + txv) % g.nx;
    const int eyL = (ey0 - 1 + g.ny) % g.ny, eyR = (ey0 + tyv) % g.ny;
    const Ix plane = (Ix)g.nx * g.ny;
    const Ix E = (Ix)g.E;

    // this thread's node
    const int el = tid / N3;
    const int node = tid - el * N3;
    const int a = el % TX, b = el / TX;
    const bool active = el < EPB && a < txv && b < tyv;
    const int i = node % N, j = (node / N) % N, k = node / N2;

    // slot of layer L: (L - z0 + 1) mod 3
    auto slot_of = [&](int L) { return slots + ((L - z0 + 1) % 3) * CT::QSLOT; };
    auto zmod = [&](int L) { return (L % g.nz + g.nz) % g.nz; };

    // prologue: layers z0 - 1, z0, z0 + 1; the z interface below z0
    column_prefetch<N, TX, TY, Ix>(Qin, slot_of(z0 - 1), g, ex0, ey0, txv, tyv, zmod(z0 - 1));
    column_prefetch<N, TX, TY, Ix>(Qin, slot_of(z0), g, ex0, ey0, txv, tyv, zmod(z0));
    column_prefetch<N, TX, TY, Ix>(Qin, slot_of(z0 + 1), g, ex0, ey0, txv, tyv, zmod(z0 + 1));
    cp_async_wait_all();
    __syncthreads();
    // z slabs: the traces of another slab's layer, from the halo [NF][nx*ny][N^2]
    auto halo_task = [&](const void *halo, int e2, int ln, int face) {
        const Ix col = (Ix)(ex0 + e2 % TX) + (Ix)g.nx * (ey0 + e2 / TX);
        const float *h = static_cast<const float *>(halo) + col * N2 + ln;
        float *tt = sT + (size_t)e2 * TSTR + (face * NF) * N2 + ln;
#pragma unroll
        for (int n = 0; n < NF; ++n) tt[n * N2] = h[(Ix)n * plane * N2];
    };
    for (int t = tid; t < 2 * EPB * N2; t += nthr) {
        const int w = t / (EPB * N2), r = t - w * (EPB * N2);
        const int e2 = r / N2, ln = r - e2 * N2;
        if (e2 % TX >= txv || e2 / TX >= tyv) continue;
        if (w == 0 && g.zlo != nullptr && z0 == 0) halo_task(g.zlo, e2, ln, 5);
        else if (w == 0) line_task<N, TX, TY, 2>(slot_of(z0 - 1), sT, lm, lp, e2, ln, 1);
        else line_task<N, TX, TY, 2>(slot_of(z0), sT, lm, lp, e2, ln, 0);
    }
    __syncthreads();
    for (int t = tid; t < EPB * N2; t += nthr) {
        const int e2 = t / N2, pt = t - e2 * N2;
        if (e2 % TX >= txv || e2 / TX >= tyv) continue;
        const float *tt = sT + (size_t)e2 * TSTR;
        float qL[NF], qR[NF], f[NF];
#pragma unroll
        for (int n = 0; n < NF; ++n) {
            qL[n] = tt[(5 * NF + n) * N2 + pt];
            qR[n] = tt[(4 * NF + n) * N2 + pt];
        }
        lf_flux2_f<2>(qL, qR, gamma, gm1, f);
        float *zf = sZ + ((z0 & 1) * EPB + e2) * ZSTR + pt;
#pragma unroll
        for (int n = 0; n < NF; ++n) zf[n * N2] = f[n];
    }
    __syncthreads();
    if (z0 + 2 <= z1)
        column_prefetch<N, TX, TY, Ix>(Qin, slot_of(z0 + 2), g, ex0, ey0, txv, tyv, zmod(z0 + 2));

    for (int z = z0; z < z1; ++z) {
        const float *cur = slot_of(z), *nxt = slot_of(z + 1);
        const Ix e = ex0 + a + (Ix)g.nx * (ey0 + b) + plane * z;

        // B: node fluxes, line traces; the node's dQ fetched early
        float dq[NF];
        if (active) {
            if (MODE != 0 && A != 0.0f) {
#pragma unroll
                for (int n = 0; n < NF; ++n) dq[n] = dQ[((Ix)n * E + e) * N3 + node];
            }
            float q[NF];
#pragma unroll
            for (int n = 0; n < NF; ++n) q[n] = cur[(n * EPB + el) * CT::ESTR + node];
            float fx[NF], fy[NF], fz[NF];
            node_flux_f(q, gm1, fx, fy, fz);
            float *sx = sF + (size_t)el * FSTR + 0 * NF * N3 + (k * N + j) * N + i;
            float *sy = sF + (size_t)el * FSTR + 1 * NF * N3 + (k * N + i) * N + j;
            float *sz = sF + (size_t)el * FSTR + 2 * NF * N3 + (j * N + i) * N + k;
#pragma unroll
            for (int n = 0; n < NF; ++n) {
                sx[n * N3] = fx[n];
                sy[n * N3] = fy[n];
                sz[n * N3] = fz[n];
            }
        }
        for (int t = tid; t < CT::LINE_TASKS; t += nthr) {
            const int w = t / (EPB * N2), r = t - w * (EPB * N2);
            const int e2 = r / N2, ln = r - e2 * N2;
            if (e2 % TX >= txv || e2 / TX >= tyv) continue;
            if (w == 0) line_task<N, TX, TY, 0>(cur, sT, lm, lp, e2, ln, 2);
            else if (w == 1) line_task<N, TX, TY, 1>(cur, sT, lm, lp, e2, ln, 2);
            else if (w == 2) line_task<N, TX, TY, 2>(cur, sT, lm, lp, e2, ln, 1);
            else if (g.zhi != nullptr && z == g.nz - 1) halo_task(g.zhi, e2, ln, 4);
            else line_task<N, TX, TY, 2>(nxt, sT, lm, lp, e2, ln, 0);
        }
        __syncthreads();

        // D: interface fluxes, each interface of the layer once
        for (int t = tid; t < CT::XT + CT::YT + CT::ZT; t += nthr) {
            if (t < CT::XT) {
                // interface index slowest, so that a warp shares its source
                const int ai = t / (TY * N2), r = t - ai * (TY * N2);
                const int row = r / N2, pt = r - row * N2;
                if (ai > txv || row >= tyv) continue;
                const Ix er = (Ix)g.nx * (ey0 + row) + plane * z;
                plane_interface<N, TX, TY, 0, Ix>(Qin, sT, sH, g, lm, lp, gamma, gm1, ai, row, txv,
                                              exL + er, exR + er, pt);
            } else if (t < CT::XT + CT::YT) {
                const int u = t - CT::XT;
                const int ai = u / (TX * N2), r = u - ai * (TX * N2);
                const int cx = r / N2, pt = r - cx * N2;
                if (ai > tyv || cx >= txv) continue;
                const Ix ec = ex0 + cx + plane * z;
                plane_interface<N, TX, TY, 1, Ix>(Qin, sT, sH, g, lm, lp, gamma, gm1, ai, cx, tyv,
                                                  ec + (Ix)g.nx * eyL, ec + (Ix)g.nx * eyR, pt);
            } else {
                const int u = t - CT::XT - CT::YT;
                const int e2 = u / N2, pt = u - e2 * N2;
                if (e2 % TX >= txv || e2 / TX >= tyv) continue;
                const float *tt = sT + (size_t)e2 * TSTR;
                float qL[NF], qR[NF], f[NF];
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    qL[n] = tt[(5 * NF + n) * N2 + pt];
                    qR[n] = tt[(4 * NF + n) * N2 + pt];
                }
                lf_flux2_f<2>(qL, qR, gamma, gm1, f);
                float *zf = sZ + (((z + 1) & 1) * EPB + e2) * ZSTR + pt;
#pragma unroll
                for (int n = 0; n < NF; ++n) zf[n * N2] = f[n];
            }
        }
        __syncthreads();

        // G: derivative, lift, update
        if (active) {
            const int px = k * N + j, py = k * N + i, pz = j * N + i;
            const float *h = sH + (size_t)el * HSTR;
            const float *f = sF + (size_t)el * FSTR;
            const float *zm = sZ + ((z & 1) * EPB + el) * ZSTR;
            const float *zp = sZ + (((z + 1) & 1) * EPB + el) * ZSTR;
            float dx[N], dy[N], dz[N];
            load_line<N>(sOp + 0 * N2 + i * N, dx);
            load_line<N>(sOp + 1 * N2 + j * N, dy);
            load_line<N>(sOp + 2 * N2 + k * N, dz);
            const float *Lm = sOp + 3 * N2, *Lp = Lm + 3 * N;
            const float lmx = Lm[i], lmy = Lm[N + j], lmz = Lm[2 * N + k];
            const float lpx = Lp[i], lpy = Lp[N + j], lpz = Lp[2 * N + k];
#pragma unroll
            for (int n = 0; n < NF; ++n) {
                float vx[N], vy[N], vz[N];
                load_line<N>(f + 0 * NF * N3 + n * N3 + (k * N + j) * N, vx);
                load_line<N>(f + 1 * NF * N3 + n * N3 + (k * N + i) * N, vy);
                load_line<N>(f + 2 * NF * N3 + n * N3 + (j * N + i) * N, vz);
                // packed pairs, explicitly rounded: every instantiation (rhs,
                // stage, a step's last stage) gives the same floats
                float2 a2 = f2(0.0f, 0.0f);
                a2 = dot2_acc<N>(dx, vx, a2);
                a2 = dot2_acc<N>(dy, vy, a2);
                a2 = dot2_acc<N>(dz, vz, a2);
                const float2 hx = *reinterpret_cast<const float2 *>(h + ((0 * NF + n) * N2 + px) * 2);
                const float2 hy = *reinterpret_cast<const float2 *>(h + ((1 * NF + n) * N2 + py) * 2);
                a2 = __ffma2_rn(f2(lmx, -lpx), hx, a2);
                a2 = __ffma2_rn(f2(lmy, -lpy), hy, a2);
                a2 = __ffma2_rn(f2(lmz, -lpz), f2(zm[n * N2 + pz], zp[n * N2 + pz]), a2);
                const float acc = __fadd_rn(a2.x, a2.y);
                const Ix o = ((Ix)n * E + e) * N3 + node;
                if (MODE == 0) {
                    Out[o] = acc;
                } else {
                    const float d = __fmaf_rn(dtr, acc, A == 0.0f ? 0.0f : __fmul_rn(A, dq[n]));
                    if (MODE == 1) dQ[o] = d;
                    Out[o] = __fmaf_rn(B, d, cur[(n * EPB + el) * CT::ESTR + node]);
                }
            }
        }
        // the slot of layer z is free once every thread is past G
        cp_async_wait_all();
        __syncthreads();
        if (z + 3 <= z1)
            column_prefetch<N, TX, TY, Ix>(Qin, slots + ((z - z0 + 1) % 3) * CT::QSLOT, g, ex0, ey0,
                                       txv, tyv, zmod(z + 3));
    }
}
