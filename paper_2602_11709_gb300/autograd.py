"""torch.autograd.Function over the broadened-pattern kernels.

    y = broadened_pattern(frac, B, lattice, fixed, opts, grid, handle)

frac [n_atoms, 3], B [n_atoms] and lattice [n_struct, 6] (float64, CUDA) are
differentiable; `fixed` holds the non-differentiable part of the batch
(atom offsets, element numbers, occupancies, scattering coefficients). The
forward pass runs xrd_pattern_broadened, the backward pass xrd_pattern_grad on
the same workspace (the reflection set of the forward pass is held fixed).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import xrd


@dataclass
class FixedBatch:
    atom_off: torch.Tensor  # int64 [n_struct + 1]
    Z: torch.Tensor         # int16 [n_atoms]
    occ: torch.Tensor       # float64 [n_atoms]
    coef: torch.Tensor      # float64 [zmax + 1, 4, 2]
    zmax: int

    @staticmethod
    def from_host(b, device="cuda"):
        d = xrd.DeviceBatch.from_host(b, device)
        return FixedBatch(d.atom_off, d.Z, d.occ, d.coef, d.zmax)


def _device_batch(frac, B, lattice, fx: FixedBatch) -> xrd.DeviceBatch:
    return xrd.DeviceBatch(int(lattice.shape[0]), fx.zmax, int(frac.shape[0]), lattice, fx.atom_off, frac, fx.Z,
                           fx.occ, B, fx.coef)


class BroadenedPattern(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frac, B, lattice, fixed: FixedBatch, opts, grid, handle: xrd.Handle):
        frac_c = frac.detach().contiguous().to(torch.float64)
        B_c = B.detach().contiguous().to(torch.float64)
        lat_c = lattice.detach().contiguous().to(torch.float64)
        db = _device_batch(frac_c, B_c, lat_c, fixed)
        co = xrd.make_opts(opts, "fp32_phasefix")
        cg = xrd.make_grid(grid)
        sz = handle.query_sizes(db, co)
        ws = xrd.workspace(sz.ws_grad_bytes, frac.device)
        n = db.n_struct
        y = torch.empty(n, int(grid.n_pts), dtype=torch.float32, device=frac.device)
        status = torch.zeros(n, dtype=torch.int32, device=frac.device)
        totals = torch.zeros(4, dtype=torch.int64, device=frac.device)
        handle.pattern_broadened(db, co, cg, y, status, totals, ws)
        ctx.state = (db, co, cg, ws, handle, status)
        ctx.dtypes = (frac.dtype, B.dtype, lattice.dtype)
        return y

    @staticmethod
    def backward(ctx, gy):
        db, co, cg, ws, handle, _ = ctx.state
        gy = gy.detach().contiguous().to(torch.float32)
        dev = gy.device
        d_frac = torch.empty(db.n_atoms, 3, dtype=torch.float32, device=dev)
        d_B = torch.empty(db.n_atoms, dtype=torch.float32, device=dev)
        d_lat = torch.empty(db.n_struct, 6, dtype=torch.float32, device=dev)
        handle.pattern_grad(db, co, cg, gy, d_frac, d_B, d_lat, ws)
        tf, tb, tl = ctx.dtypes
        return d_frac.to(tf), d_B.to(tb), d_lat.to(tl), None, None, None, None


def broadened_pattern(frac, B, lattice, fixed: FixedBatch, opts, grid, handle: xrd.Handle):
    return BroadenedPattern.apply(frac, B, lattice, fixed, opts, grid, handle)
