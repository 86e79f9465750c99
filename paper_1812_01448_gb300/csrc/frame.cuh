// PML frame: per-thread updates of the frame's sides, interface edges and cells, run by extra
// blocks of the plain step's two kernels (kernels_step.cu).  Layout in device.cuh (FrameDev).
//
// The frame is a Yee grid of square cells of side h.  Its unknowns are circulations like the
// mesh's: U = h E on the cell sides, B at the cell centres, split as B = Bx + By (Berenger):
//   side along +x at height J:   U = aH[J] U + bH[J] (B_above - B_below)
//   side along +y at column I:   U = aV[I] U + bV[I] (B_left - B_right)
//   cell (I, J):                 Bx = axc[I] Bx - bxc[I] (U_right - U_left)
//                                By = ayc[J] By - byc[J] (U_bottom - U_top)
// with a = (1 - sigma dt/2) / (1 + sigma dt/2), b = dt / (1 + sigma dt/2) on sides and
// (dt / h^2) / (1 + sigma dt/2) on cells: the trapezoidal decay of the split-field PML, sigma
// taken at each field's position.  The mesh's outer edges (interface edges) couple a triangle
// and a frame cell: U += dt |e| / d (B_R - B_L) in the mesh edge's direction, their values kept
// after the zero slot of the U array the triangles' edge codes point into: the mesh's, or, in
// blocked stepping, that of the region stepped with the frame.
// Every operation is explicitly rounded.
#pragma once

#include "device.cuh"

namespace ue {

template <typename T>
struct Tab {
    const T *aH, *bH, *aV, *bV, *axc, *bxc, *ayc, *byc;
};

template <typename T>
__device__ __forceinline__ Tab<T> tabs(const FrameDev& f) {
    Tab<T> t;
    t.aH = (const T*)f.tab;
    t.bH = t.aH + f.NY + 1;
    t.aV = t.bH + f.NY + 1;
    t.bV = t.aV + f.NX + 1;
    t.axc = t.bV + f.NX + 1;
    t.bxc = t.axc + f.NX;
    t.ayc = t.bxc + f.NX;
    t.byc = t.ayc + f.NY;
    return t;
}

template <typename T>
__device__ __forceinline__ T cellB(const FrameDev& f, int64_t c) {
    return rn_add(((const T*)f.Bx)[c], ((const T*)f.By)[c]);
}

// E half-step of the frame for thread t: t < n_fc updates cell t's bottom and left sides (those
// that are frame unknowns), n_fc <= t < n_fc + n_if interface edge t - n_fc (reads B, writes U).
template <typename T>
__device__ __forceinline__ void frame_edge_thread(const FrameDev& f, const T* __restrict__ B,
                                                  T* __restrict__ U, int64_t t) {
    if (t < f.n_fc) {
        const Tab<T> tb = tabs<T>(f);
        int I, J;
        frame_ij(f, t, I, J);
        const T Bc = cellB<T>(f, t);
        if (frame_is_cell(f, I, J - 1)) {   // bottom side: R = this cell (above), L = below
            const T Bb = cellB<T>(f, frame_cell(f, I, J - 1));
            T* u = (T*)f.H + (int64_t)J * f.NX + I;
            *u = rn_fma(tb.aH[J], *u, rn_mul(tb.bH[J], rn_sub(Bc, Bb)));
        }
        if (frame_is_cell(f, I - 1, J)) {   // left side: R = left cell, L = this cell
            const T Bl = cellB<T>(f, frame_cell(f, I - 1, J));
            T* u = (T*)f.V + (int64_t)J * (f.NX + 1) + I;
            *u = rn_fma(tb.aV[I], *u, rn_mul(tb.bV[I], rn_sub(Bl, Bc)));
        }
    } else if (t < f.n_fc + f.n_if) {
        const int64_t k = t - f.n_fc;
        const T Bc = cellB<T>(f, f.icell[k]);
        const int32_t code = f.itri[k];
        const T Bt = B[code >= 0 ? code : ~code];
        const T diff = code >= 0 ? rn_sub(Bt, Bc) : rn_sub(Bc, Bt);
        T* u = U + f.u_off + k;
        *u = rn_fma(((const T*)f.icU)[k], diff, *u);
    }
}

// A cell side's counter-clockwise contribution to the cell's circulation: frame sides in their
// +x / +y direction with sign sgn, interface sides in the mesh edge's direction with the cell's
// own sign (+1 when the cell is R of the edge, i.e. the triangle is L), PEC sides 0.
template <typename T>
__device__ __forceinline__ T side_h(const FrameDev& f, const T* __restrict__ U, int I, int J, int Jo,
                                    T sgn, int64_t k_if) {
    if (frame_is_cell(f, I, Jo)) {
        const T u = ((const T*)f.H)[(int64_t)J * f.NX + I];
        return sgn > T(0) ? u : -u;
    }
    if (k_if >= 0) {
        const T u = U[f.u_off + k_if];
        return f.itri[k_if] >= 0 ? -u : u;
    }
    return T(0);
}
template <typename T>
__device__ __forceinline__ T side_v(const FrameDev& f, const T* __restrict__ U, int I, int J, int Io,
                                    T sgn, int64_t k_if) {
    if (frame_is_cell(f, Io, J)) {
        const T u = ((const T*)f.V)[(int64_t)J * (f.NX + 1) + I];
        return sgn > T(0) ? u : -u;
    }
    if (k_if >= 0) {
        const T u = U[f.u_off + k_if];
        return f.itri[k_if] >= 0 ? -u : u;
    }
    return T(0);
}

// B half-step of frame cell c (reads U of its sides and interface edges, writes its Bx, By).
template <typename T>
__device__ __forceinline__ void frame_cell_thread(const FrameDev& f, const T* __restrict__ U, int64_t c) {
    if (c >= f.n_fc) return;
    const Tab<T> tb = tabs<T>(f);
    int I, J;
    frame_ij(f, c, I, J);
    const bool in_x = I >= f.W && I < f.W + f.nx, in_y = J >= f.W && J < f.W + f.ny;
    // interface edges on this cell's sides: the mesh lies above (bottom row under it), below,
    // to the right or to the left
    const int64_t k_top = (in_x && J == f.W - 1) ? (I - f.W) : -1;
    const int64_t k_bot = (in_x && J == f.W + f.ny) ? f.nx + (I - f.W) : -1;
    const int64_t k_right = (in_y && I == f.W - 1) ? 2 * (int64_t)f.nx + (J - f.W) : -1;
    const int64_t k_left = (in_y && I == f.W + f.nx) ? 2 * (int64_t)f.nx + f.ny + (J - f.W) : -1;
    const T bottom = side_h<T>(f, U, I, J, J - 1, T(1), k_bot);
    const T top = side_h<T>(f, U, I, J + 1, J + 1, T(-1), k_top);
    const T left = side_v<T>(f, U, I, J, I - 1, T(-1), k_left);
    const T right = side_v<T>(f, U, I + 1, J, I + 1, T(1), k_right);
    const T cx = rn_add(right, left), cy = rn_add(bottom, top);
    T* bx = (T*)f.Bx + c;
    T* by = (T*)f.By + c;
    *bx = rn_sub(rn_mul(tb.axc[I], *bx), rn_mul(tb.bxc[I], cx));
    *by = rn_sub(rn_mul(tb.ayc[J], *by), rn_mul(tb.byc[J], cy));
}

}  // namespace ue
