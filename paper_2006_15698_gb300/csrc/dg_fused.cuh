// dg_fused.cuh -- the float form's fused single-pass RK stage on element
// tiles (faces + volume + lift + update in one kernel) for one mesh, and the
// time-step reduction of a batch of independent meshes.  Included by
// dg_kernels.cuh.
//
// For the float form the stage is bound by DRAM traffic and instruction
// issue, not by a narrow pipe, so one kernel does all of it: a CTA stages a
// tile of elements' states and fluxes in shared memory, computes the
// Lax-Friedrichs flux on all six faces of each of its elements (the
// neighbour's trace is interpolated from the neighbour's face-normal node
// lines, read through L2, or from shared memory when the neighbour is in the
// same tile), then the derivative, lift and update.  Each interface flux is
// evaluated by both adjacent tiles from bitwise-identical inputs in the same
// operation order, so both see the same value and discrete conservation holds
// as in the two-kernel form.  DRAM traffic per stage is Q read, dQ
// read/written and Q' written: the output goes to a second state buffer,
// because neighbouring tiles still read the input state.
//
// A tile is TX x TY elements of one z layer (x fastest); the shape per
// polynomial order is chosen by the autotuner among the variants below.
#pragma once

// (included inside namespace dg)

// single-instruction float approximations (PTX rcp.approx / sqrt.approx,
// relative error of order 2^-23, the float form's own rounding level)
__device__ __forceinline__ float fast_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fast_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Wave-speed sum sum_d (|u_d| + c) of a float node, in float (the precision
// of the state itself); false for rho <= 0, p <= 0 or NaN.  Every operation
// explicitly rounded in a fixed order (no contraction), so every kernel that
// evaluates it gets the same float; callers keep the maximum in float
// (conversion to double is exact and monotonic) and the time step in double.
__device__ __forceinline__ bool node_speed_f(float r, float mx, float my, float mz, float E,
                                             float g, float &s)
{
    const float rinv = __fdiv_rn(1.0f, r);
    const float u = __fmul_rn(mx, rinv), v = __fmul_rn(my, rinv), w = __fmul_rn(mz, rinv);
    const float uu = __fadd_rn(__fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v)), __fmul_rn(w, w));
    const float p = __fmul_rn(g - 1.0f, __fsub_rn(E, __fmul_rn(__fmul_rn(0.5f, r), uu)));
    if (!(r > 0.0f) || !(p > 0.0f)) return false;
    const float c = __fsqrt_rn(__fmul_rn(__fmul_rn(g, p), rinv));
    s = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(u), c), __fadd_rn(fabsf(v), c)), __fadd_rn(fabsf(w), c));
    return true;
}

template <int DIR>
__device__ __forceinline__ void normal_flux_f(const float q[NF], float gamma, float gm1,
                                              float f[NF], float &speed)
{
    const float rinv = fast_rcp(q[0]);
    const float mm = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    const float p = gm1 * (q[4] - 0.5f * mm * rinv);
    const float mn = q[1 + DIR];
    const float un = mn * rinv;
    f[0] = mn;
    f[1] = q[1] * un + (DIR == 0 ? p : 0.0f);
    f[2] = q[2] * un + (DIR == 1 ? p : 0.0f);
    f[3] = q[3] * un + (DIR == 2 ? p : 0.0f);
    f[4] = (q[4] + p) * un;
    speed = fabsf(un) + fast_sqrt(gamma * p * rinv);
}

// N consecutive floats; vector loads when the line is 8- or 16-byte aligned
// (N even: every line starts at a multiple of N floats from an aligned base)
template <int N>
__device__ __forceinline__ void load_line(const float *p, float v[N])
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int a = 0; a < N; a += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y; v[a + 2] = t.z; v[a + 3] = t.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int a = 0; a < N; a += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int a = 0; a < N; ++a) v[a] = p[a];
    }
}

// Trace of an element on a face in direction DIR at node line (t1, t2):
// sum_c l[c] Q(node c along DIR), from `src` (the element's field planes at
// plane stride `pstride`); the same arithmetic for shared and global sources.
// Ix: index type of the state arrays (32-bit when every offset fits).
template <int N, int DIR, typename Ix>
__device__ __forceinline__ void line_trace(const float *src, Ix pstride, int base,
                                           const float *l, float q[NF])
{
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? N : N * N);
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        float v[N];
        if constexpr (DIR == 0) {
            load_line<N>(src + n * pstride + base, v);
        } else {
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = src[n * pstride + base + c * stride];
        }
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < N; ++c) s += l[c] * v[c];
        q[n] = s;
    }
}

// ---------------------------------------------------------------------------
// tile shapes
// ---------------------------------------------------------------------------

// Variants per N (= p + 1): (TX, TY) elements per tile.
template <int N, int V>
struct TileShape;
template <> struct TileShape<1, 0> { static constexpr int TX = 128, TY = 1; };
template <> struct TileShape<1, 1> { static constexpr int TX = 256, TY = 1; };
template <> struct TileShape<2, 0> { static constexpr int TX = 32, TY = 1; };
template <> struct TileShape<2, 1> { static constexpr int TX = 16, TY = 2; };
template <> struct TileShape<2, 2> { static constexpr int TX = 8, TY = 4; };
template <> struct TileShape<3, 0> { static constexpr int TX = 9, TY = 1; };
template <> struct TileShape<3, 1> { static constexpr int TX = 3, TY = 3; };
template <> struct TileShape<4, 0> { static constexpr int TX = 4, TY = 1; };
template <> struct TileShape<4, 1> { static constexpr int TX = 2, TY = 2; };
template <> struct TileShape<5, 0> { static constexpr int TX = 2, TY = 1; };
template <> struct TileShape<5, 1> { static constexpr int TX = 1, TY = 1; };
template <> struct TileShape<6, 0> { static constexpr int TX = 1, TY = 1; };
template <> struct TileShape<7, 0> { static constexpr int TX = 1, TY = 1; };
constexpr int kTileVariants[8] = {0, 2, 3, 2, 2, 2, 1, 1};  // per N

template <int N, int TX, int TY>
struct FusedTile {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int EPB = TX * TY;
    static constexpr int THREADS = ((EPB * N3 + 31) / 32) * 32;
    // face tasks: six faces, each a warp-aligned segment of EPB N^2 points
    static constexpr int SEGF = ((EPB * N2 + 31) / 32) * 32;
    // per-element strides in shared memory, padded to 16 (mod 32) floats so
    // that two elements touched by one warp fall into different bank halves
    static constexpr int pad16(int x) { return x + ((16 - x % 32) + 32) % 32; }
    static constexpr int FSTR = pad16(3 * NF * N3);      // fluxes [3][NF][N3], direction-major
    static constexpr int QSTR = pad16(NF * N3);          // state [NF][N3]
    static constexpr int HSTR = pad16(3 * NF * N2 * 2);  // face fluxes [3][NF][N2][(-,+)]
    // operators D[3][N][N], Lm[3][N], Lp[3][N] (read by every thread at its own
    // node index, so from shared memory rather than the constant bank)
    static constexpr int OPSF = ((3 * N2 + 6 * N + 3) / 4) * 4;
    // fluxes, state, face fluxes, operators (floats), then the neighbour table [EPB][6]
    static constexpr size_t FLOATS = (size_t)EPB * (FSTR + QSTR + HSTR) + OPSF;
    static constexpr size_t BYTES = ((FLOATS * sizeof(float) + 15) / 16) * 16 + EPB * 6 * 8;
};


// ---------------------------------------------------------------------------
// one tile of the fused stage
// ---------------------------------------------------------------------------

// Neighbour table entry: >= 0 a global element index, < 0 the in-tile index
// -(local + 1) of a neighbour that sits in the same tile.
template <int N, int DIR, int TX, int TY, typename Ix>
__device__ __forceinline__ void fused_face(const float *__restrict__ Qin, const float *sQ,
                                           float *sH, const long long *sNb, const Ops<float> &T,
                                           Ix E, int el, int side, int pt)
{
    using FT = FusedTile<N, TX, TY>;
    constexpr int N2 = N * N, N3 = N * N * N;
    const int t1 = pt % N, t2 = pt / N;
    const int base = DIR == 0 ? (t2 * N + t1) * N : (DIR == 1 ? t2 * N2 + t1 : t2 * N + t1);
    const Ix nb = (Ix)sNb[el * 6 + 2 * DIR + side];
    // own trace at the face's end of the element, the neighbour's at the other end
    float qo[NF], qn[NF];
    line_trace<N, DIR, Ix>(sQ + (size_t)el * FT::QSTR, (Ix)N3, base, side ? T.lp : T.lm, qo);
    if (nb < 0)
        line_trace<N, DIR, Ix>(sQ + (size_t)(-nb - 1) * FT::QSTR, (Ix)N3, base, side ? T.lm : T.lp, qn);
    else
        line_trace<N, DIR, Ix>(Qin + nb * N3, E * N3, base, side ? T.lm : T.lp, qn);
    // left and right states by value selects (a pointer select between two
    // local arrays would force them out of registers)
    float qL[NF], qR[NF];
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        qL[n] = side ? qo[n] : qn[n];
        qR[n] = side ? qn[n] : qo[n];
    }
    float fL[NF], fR[NF], sL, sR;
    normal_flux_f<DIR>(qL, T.gamma, T.gm1, fL, sL);
    normal_flux_f<DIR>(qR, T.gamma, T.gm1, fR, sR);
    const float lam = fmaxf(sL, sR);
    // (-, +) pair of the direction's two faces at this face point
    float *h = sH + (size_t)el * FT::HSTR + (DIR * NF * N2 + pt) * 2 + side;
#pragma unroll
    for (int n = 0; n < NF; ++n) h[n * N2 * 2] = (fL[n] + fR[n]) - lam * (qR[n] - qL[n]);
}

// One tile of the stage with blockDim.x >= TX*TY*N^3 threads (one per node;
// extra threads only help with the face tasks).  MODE 0 writes the rhs to
// Out, MODE 1 the LSERK stage update (dQ <- A dQ + dt R, Out <- Qin + B dQ),
// MODE 2 a step's last stage, whose dQ no later stage reads: only
// Out <- Qin + B (A dQ + dt R), dQ left as it was.
// Ends with a barrier, so a persistent caller may reuse `smem` at once.
// Ix: index type of the state arrays (32-bit when every offset fits).
template <int N, int TX, int TY, int MODE, typename Ix = long long>
__device__ __forceinline__ void fused_tile(const float *__restrict__ Qin, float *__restrict__ Out,
                                           float *__restrict__ dQ, const Ops<float> &T,
                                           const Geo &g, long long tile, float A, float B,
                                           float dtr, unsigned char *smem)
{
    using FT = FusedTile<N, TX, TY>;
    constexpr int N2 = FT::N2, N3 = FT::N3, EPB = FT::EPB, SEGF = FT::SEGF;
    constexpr int FSTR = FT::FSTR, QSTR = FT::QSTR, HSTR = FT::HSTR;
    float *sF = reinterpret_cast<float *>(smem);  // [EPB][FSTR]
    float *sQ = sF + EPB * FSTR;                  // [EPB][QSTR]
    float *sH = sQ + EPB * QSTR;                  // [EPB][HSTR]
    float *sOp = sH + EPB * HSTR;                 // D[3][N][N], Lm[3][N], Lp[3][N]
    long long *sNb = reinterpret_cast<long long *>(smem + (FT::BYTES - EPB * 6 * 8));

    // tile -> element coordinates of its corner
    const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY;
    const int bx = (int)(tile % ntx);
    const int by = (int)((tile / ntx) % nty);
    const int bz = (int)(tile / ((long long)ntx * nty));
    const int ex0 = bx * TX, ey0 = by * TY;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int el = tid / N3;
    const int node = tid - el * N3;
    const int a = el % TX, b = el / TX;
    const bool in_tile = el < EPB;
    const bool active = in_tile && ex0 + a < g.nx && ey0 + b < g.ny;
    const Ix E = (Ix)g.E;
    const Ix e = (Ix)(ex0 + a) + (Ix)g.nx * ((ey0 + b) + (Ix)g.ny * bz);
    const int i = node % N, j = (node / N) % N, k = node / N2;

    for (int t = tid; t < EPB * 6; t += nthr) {  // the six neighbours of every element of the tile
        const int te = t / 6, f = t - te * 6;
        const int ta = te % TX, tb = te / TX;
        const int d = f >> 1, s = (f & 1) ? 1 : -1;
        int cx = ex0 + ta, cy = ey0 + tb, cz = bz;
        long long nb = 0;
        if (cx < g.nx && cy < g.ny) {
            if (d == 0) cx = (cx + s + g.nx) % g.nx;
            else if (d == 1) cy = (cy + s + g.ny) % g.ny;
            else cz = (cz + s + g.nz) % g.nz;
            const int la = cx - ex0, lb = cy - ey0;
            if (cz == bz && la >= 0 && la < TX && lb >= 0 && lb < TY)
                nb = -(long long)(lb * TX + la) - 1;
            else
                nb = (long long)((Ix)cx + (Ix)g.nx * (cy + (Ix)g.ny * cz));
        }
        sNb[t] = nb;
    }

    for (int t = tid; t < 3 * N2 + 6 * N; t += nthr) {
        float v;
        if (t < 3 * N2) v = T.D[t / N2][(t % N2) / N][t % N];
        else if (t < 3 * N2 + 3 * N) v = T.Lm[(t - 3 * N2) / N][(t - 3 * N2) % N];
        else v = T.Lp[(t - 3 * N2 - 3 * N) / N][(t - 3 * N2 - 3 * N) % N];
        sOp[t] = v;
    }

    float q[NF];
    if (active) {
#pragma unroll
        for (int n = 0; n < NF; ++n) {
            q[n] = Qin[((Ix)n * E + e) * N3 + node];
            sQ[el * QSTR + n * N3 + node] = q[n];
        }
        const float rinv = fast_rcp(q[0]);
        const float u = q[1] * rinv, v = q[2] * rinv, w = q[3] * rinv;
        const float p = T.gm1 * (q[4] - 0.5f * (q[1] * u + q[2] * v + q[3] * w));
        const float ep = q[4] + p;
        // direction-major node order: the line a contraction reads is contiguous
        float *sx = sF + (size_t)el * FSTR + 0 * NF * N3 + (k * N + j) * N + i;
        float *sy = sF + (size_t)el * FSTR + 1 * NF * N3 + (k * N + i) * N + j;
        float *sz = sF + (size_t)el * FSTR + 2 * NF * N3 + (j * N + i) * N + k;
        sx[0 * N3] = q[1];
        sx[1 * N3] = q[1] * u + p;
        sx[2 * N3] = q[2] * u;
        sx[3 * N3] = q[3] * u;
        sx[4 * N3] = ep * u;
        sy[0 * N3] = q[2];
        sy[1 * N3] = q[1] * v;
        sy[2 * N3] = q[2] * v + p;
        sy[3 * N3] = q[3] * v;
        sy[4 * N3] = ep * v;
        sz[0 * N3] = q[3];
        sz[1 * N3] = q[1] * w;
        sz[2 * N3] = q[2] * w;
        sz[3 * N3] = q[3] * w + p;
        sz[4 * N3] = ep * w;
    }
    __syncthreads();

    // the six faces of every element of the tile, face-major so that a warp
    // works on one (direction, side)
    for (int t = tid; t < 6 * SEGF; t += nthr) {
        const int face = t / SEGF;
        const int r = t - face * SEGF;
        if (r >= EPB * N2) continue;
        const int el2 = r / N2;
        const int pt = r - el2 * N2;
        if (ex0 + el2 % TX >= g.nx || ey0 + el2 / TX >= g.ny) continue;
        const int side = face & 1;
        if (face < 2) fused_face<N, 0, TX, TY, Ix>(Qin, sQ, sH, sNb, T, E, el2, side, pt);
        else if (face < 4) fused_face<N, 1, TX, TY, Ix>(Qin, sQ, sH, sNb, T, E, el2, side, pt);
        else fused_face<N, 2, TX, TY, Ix>(Qin, sQ, sH, sNb, T, E, el2, side, pt);
    }
    __syncthreads();

    if (active) {
        const int px = k * N + j, py = k * N + i, pz = j * N + i;
        const float *h = sH + (size_t)el * HSTR;
        const float *f = sF + (size_t)el * FSTR;
        float dx[N], dy[N], dz[N];
        load_line<N>(sOp + 0 * N2 + i * N, dx);
        load_line<N>(sOp + 1 * N2 + j * N, dy);
        load_line<N>(sOp + 2 * N2 + k * N, dz);
        const float *lm = sOp + 3 * N2, *lp = lm + 3 * N;
        const float lmx = lm[i], lmy = lm[N + j], lmz = lm[2 * N + k];
        const float lpx = lp[i], lpy = lp[N + j], lpz = lp[2 * N + k];
#pragma unroll
        for (int n = 0; n < NF; ++n) {
            float vx[N], vy[N], vz[N];
            load_line<N>(f + 0 * NF * N3 + n * N3 + (k * N + j) * N, vx);
            load_line<N>(f + 1 * NF * N3 + n * N3 + (k * N + i) * N, vy);
            load_line<N>(f + 2 * NF * N3 + n * N3 + (j * N + i) * N, vz);
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < N; ++c) acc = __fmaf_rn(dx[c], vx[c], acc);
#pragma unroll
            for (int c = 0; c < N; ++c) acc = __fmaf_rn(dy[c], vy[c], acc);
#pragma unroll
            for (int c = 0; c < N; ++c) acc = __fmaf_rn(dz[c], vz[c], acc);
            // lift: one (-, +) pair of face fluxes per direction
            const float2 hx = *reinterpret_cast<const float2 *>(h + ((0 * NF + n) * N2 + px) * 2);
            const float2 hy = *reinterpret_cast<const float2 *>(h + ((1 * NF + n) * N2 + py) * 2);
            const float2 hz = *reinterpret_cast<const float2 *>(h + ((2 * NF + n) * N2 + pz) * 2);
            // explicitly rounded: every instantiation (rhs, stage, a step's
            // last stage) gives the same floats
            acc = __fmaf_rn(-lpx, hx.y, __fmaf_rn(lmx, hx.x, acc));
            acc = __fmaf_rn(-lpy, hy.y, __fmaf_rn(lmy, hy.x, acc));
            acc = __fmaf_rn(-lpz, hz.y, __fmaf_rn(lmz, hz.x, acc));

            const Ix o = ((Ix)n * E + e) * N3 + node;
            if (MODE == 0) {
                Out[o] = acc;
            } else {
                const float d = __fmaf_rn(dtr, acc, A == 0.0f ? 0.0f : __fmul_rn(A, dQ[o]));
                if (MODE == 1) dQ[o] = d;
                Out[o] = __fmaf_rn(B, d, q[n]);
            }
        }
    }
    __syncthreads();
}

// one mesh: one tile per CTA
// (at least 1280 resident threads per SM: the tile's phases are separated by
// barriers, and other CTAs' warps fill the gaps)
template <int N, int V, int MODE, typename Ix>
__global__ void __launch_bounds__(FusedTile<N, TileShape<N, V>::TX, TileShape<N, V>::TY>::THREADS,
                                  1280 / FusedTile<N, TileShape<N, V>::TX, TileShape<N, V>::TY>::THREADS)
    fused_stage_kernel(const float *__restrict__ Qin, float *__restrict__ Out,
                       float *__restrict__ dQ, const Ops<float> T, const Geo g, float A, float B,
                       const double *__restrict__ dt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const float dtr = MODE != 0 ? (float)(*dt) : 0.0f;
    fused_tile<N, TileShape<N, V>::TX, TileShape<N, V>::TY, MODE, Ix>(Qin, Out, dQ, T, g,
                                                                       blockIdx.x, A, B, dtr,
                                                                       smem_raw);
}

// ---------------------------------------------------------------------------
// batches: the time-step reduction over many independent meshes (their
// stages run batched_line_kernel, dg_lines.cuh)
// ---------------------------------------------------------------------------

#define DG_FOR_EACH_CODE(X) \
    X(1, 0) X(1, 1) X(2, 0) X(2, 1) X(2, 2) X(3, 0) X(3, 1) X(4, 0) X(4, 1) X(5, 0) X(5, 1) \
    X(6, 0) X(7, 0)

// Lambda of the shared instances of a batch: work item k covers the nodes
// [begin, end) of one instance (equal ranges of at most kLambdaNodes); a CTA
// takes items in turn, evaluates the node speeds in float (node_speed_f, as
// cfl_kernel for a float state), keeps their maximum in float and merges it
// into the instance's Lambda slot as a double (bit patterns of non-negative
// doubles; NaN, above every finite value, for a bad node).
static __global__ void __launch_bounds__(256)
    batched_lambda_kernel(const LambdaItem *__restrict__ items, int nitems,
                          const InstDev *__restrict__ inst, int parity, int *err)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const LambdaItem item = items[it];
        const InstDev &d = inst[item.inst];
        const float *Q = parity == 0 ? d.Q : d.Qt;
        const long long pl = d.g.E * (long long)((d.g.p + 1) * (d.g.p + 1) * (d.g.p + 1));
        const float gf = (float)d.g.gamma;
        float mf = 0.0f;
        bool bad = false;
        for (long long t = item.begin + threadIdx.x; t < item.end; t += blockDim.x) {
            float sp;
            if (!node_speed_f(Q[t], Q[pl + t], Q[2 * pl + t], Q[3 * pl + t], Q[4 * pl + t], gf, sp)) {
                bad = true;
                continue;
            }
            mf = fmaxf(mf, sp);
        }
        double m = (double)mf;
        if (bad) {
            atomicOr(err, 1);
            m = __longlong_as_double(0x7ff8000000000000LL);
        }
        __shared__ unsigned long long red[8];
        unsigned long long bits = (unsigned long long)__double_as_longlong(m);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long x = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = x > bits ? x : bits;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bits;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long mb = red[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mb = red[w] > mb ? red[w] : mb;
            atomicMax(d.lam_bits, mb);
        }
        __syncthreads();
    }
}

static __global__ void batched_cfl_finalize_kernel(const InstDev *__restrict__ inst, int n, double cfl)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const InstDev &d = inst[i];
        const double lam = __longlong_as_double((long long)*d.lam_bits);
        *d.dt = __ddiv_rn(__dmul_rn(cfl, d.g.hmin), __dmul_rn(2.0 * d.g.p + 1.0, lam));
        *d.lam_bits = 0ull;
    }
}
