// blocks.cuh -- device helpers over the block descriptors: cell indexing,
// the ghost/interior cells of a boundary face, buffer slots, and the lookup
// of the block that owns a work item.  Shared by the ghost-fill kernel and
// the stencil kernel's ghost push.
#pragma once

#include "sensei_internal.cuh"

namespace sensei {

__device__ __forceinline__ long long cell_index(const StateLayout &L, int i, int j, int k)
{
    return L.off + (long long)k * L.sk + (long long)j * L.sj + i;
}

// Face f (0 imin, 1 imax, 2 jmin, 3 jmax, 4 kmin, 5 kmax) of an ni x nj x nk
// block at tangential position (t1, t2): the ghost cell of layer g (1 next
// to the boundary, 2 outer) and the interior cell m cells inside (m = 0 is
// the boundary cell).
__device__ __forceinline__ void face_cells(int f, int ni, int nj, int nk, int t1, int t2, int g, int m, int &gi,
                                           int &gj, int &gk, int &mi, int &mj, int &mk)
{
    switch (f) {
    case 0: gi = -g; gj = t1; gk = t2; mi = m; mj = t1; mk = t2; break;
    case 1: gi = ni - 1 + g; gj = t1; gk = t2; mi = ni - 1 - m; mj = t1; mk = t2; break;
    case 2: gi = t1; gj = -g; gk = t2; mi = t1; mj = m; mk = t2; break;
    case 3: gi = t1; gj = nj - 1 + g; gk = t2; mi = t1; mj = nj - 1 - m; mk = t2; break;
    case 4: gi = t1; gj = t2; gk = -g; mi = t1; mj = t2; mk = m; break;
    default: gi = t1; gj = t2; gk = nk - 1 + g; mi = t1; mj = t2; mk = nk - 1 - m; break;
    }
}

// tangential coordinates of cell (i, j, k) on a face of family f >> 1
__device__ __forceinline__ void tangential(int f, int i, int j, int k, int &t1, int &t2)
{
    if (f < 2) {
        t1 = j;
        t2 = k;
    } else if (f < 4) {
        t1 = i;
        t2 = k;
    } else {
        t1 = i;
        t2 = j;
    }
}

// positions x layers of ghost-fill work on face f
__device__ __forceinline__ long long face_units(const BlockDev &B, int f)
{
    long long n1 = f < 2 ? B.nj : B.ni;
    long long n2 = f < 4 ? B.nk : B.nj;
    return n1 * n2 * 2;
}

__device__ __forceinline__ double *slot64(const BlockDev &B, double *user, int slot)
{
    return slot == SLOT_USER ? user : B.st64[slot - SLOT_ST0];
}

__device__ __forceinline__ float *slot32(const BlockDev &B, int slot) { return B.xs[slot - SLOT_X0]; }

// unit normal of boundary face f at tangential (t1, t2)
__device__ __forceinline__ void boundary_normal(const BlockDev &B, int f, int t1, int t2, double &nx, double &ny,
                                                double &nz)
{
    int i = 0, j = 0, k = 0;
    if (f < 2) {
        i = f == 0 ? 0 : B.ni;
        j = t1;
        k = t2;
    } else if (f < 4) {
        i = t1;
        j = f == 2 ? 0 : B.nj;
        k = t2;
    } else {
        i = t1;
        j = t2;
        k = f == 4 ? 0 : B.nk;
    }
    const int fam = f >> 1;
    const long long m = k * B.ml.mplane + j * B.ml.mpitch + i;
    const double *base = B.fn + (long long)(fam * 4) * B.ml.mvolume;
    nx = base[m];
    ny = base[B.ml.mvolume + m];
    nz = base[2 * B.ml.mvolume + m];
}

// the block owning work item `item` (item0 ascending), binary search
__device__ __forceinline__ int find_block_item(const BlockDev *blocks, int nb, long long item)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].item0 <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_block_bc(const BlockDev *blocks, int nb, long long unit)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].bc0 <= unit)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace sensei
