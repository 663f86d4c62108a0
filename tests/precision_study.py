"""Host-side bookkeeping of the precision study (FP32 batched path and FP64
GPU path against the FP64 oracle, per material state).

Test infrastructure: numpy only, no GPU and none of the method's
arithmetic.  It reads particle populations in the storage format of the
library and of the oracle (cell, pid, float32 momenta and weights) and
reduces them per cell and per material state.

Secondary identifiers follow the layout both sides write:
  bit 63 marker | step (19 bits) << 44 | channel (3 bits) << 41 |
  cell (24 bits) << 17 | pair j (16 bits) << 1 | sub
so one event (a Brems photon, a Trident or Bethe-Heitler e-e+ pair) is the
identifier without its last bit.
"""
from __future__ import annotations

import numpy as np

U64 = np.uint64
CHANNELS = ("brems_em", "brems_ep", "trident_em", "trident_ep", "bh")


def is_secondary(pid):
    return (np.asarray(pid, dtype=U64) >> U64(63)) == U64(1)


def secondary_step(pid):
    return ((np.asarray(pid, dtype=U64) >> U64(44)) & U64(0x7FFFF)).astype(np.int64)


def event_keys(species_list, step):
    """Sorted unique event keys (identifier >> 1) of the secondaries created
    in `step`, over the given populations."""
    keys = []
    for d in species_list:
        p = np.asarray(d["pid"], dtype=U64)
        m = is_secondary(p) & (secondary_step(p) == step)
        keys.append(p[m] >> U64(1))
    return np.unique(np.concatenate(keys)) if keys else np.zeros(0, U64)


def event_keys_all(species_list):
    """Sorted unique event keys of every live secondary, whatever its step."""
    keys = [np.asarray(d["pid"], dtype=U64)[is_secondary(d["pid"])] >> U64(1) for d in species_list]
    return np.unique(np.concatenate(keys)) if keys else np.zeros(0, U64)


def key_cell(keys):
    return ((np.asarray(keys, dtype=U64) >> U64(16)) & U64(0xFFFFFF)).astype(np.int64)


def key_channel(keys):
    return ((np.asarray(keys, dtype=U64) >> U64(40)) & U64(0x7)).astype(np.int64)


def cell_counts(d, n_cells):
    return np.bincount(np.asarray(d["cell"], dtype=np.int64), minlength=n_cells)


def pairs_per_cell(n_proj, n_targ):
    """Pairs of a cell in one group: max(N_p, N_t) when both lists are non-empty."""
    n_proj, n_targ = np.asarray(n_proj), np.asarray(n_targ)
    return np.where((n_proj > 0) & (n_targ > 0), np.maximum(n_proj, n_targ), 0)


def energy_per_cell(d, n_cells, photon):
    """FP64 sum over the cell of W E, E = gamma (rest mass included) for
    leptons and k for photons, from the stored float32 values."""
    ux, uy, uz = (np.asarray(d[k], dtype=np.float64) for k in ("ux", "uy", "uz"))
    u2 = ux * ux + uy * uy + uz * uz
    e = np.sqrt(u2) if photon else np.sqrt(1.0 + u2)
    return np.bincount(np.asarray(d["cell"], dtype=np.int64), weights=np.asarray(d["w"], np.float64) * e,
                       minlength=n_cells)


def weight_per_cell(d, n_cells):
    return np.bincount(np.asarray(d["cell"], dtype=np.int64), weights=np.asarray(d["w"], np.float64),
                       minlength=n_cells)


def photon_energies(d, step, cells_mask=None, keys=None):
    """Energies k of the photons created in `step` (optionally only in the
    cells where cells_mask is True, and only for the given event keys)."""
    p = np.asarray(d["pid"], dtype=U64)
    m = is_secondary(p) & (secondary_step(p) == step)
    if cells_mask is not None:
        m &= cells_mask[np.asarray(d["cell"], dtype=np.int64)]
    if keys is not None:
        m &= np.isin(p >> U64(1), keys)
    ux, uy, uz = (np.asarray(d[k], dtype=np.float64)[m] for k in ("ux", "uy", "uz"))
    order = np.argsort(p[m], kind="stable")
    return np.sqrt(ux * ux + uy * uy + uz * uz)[order], p[m][order]


def by_state(per_cell, state_of_cell, n_states):
    return np.bincount(state_of_cell, weights=np.asarray(per_cell, np.float64), minlength=n_states)


def rel(a, b):
    """|a/b - 1|, 0 where b == 0 and a == 0."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    out = np.zeros(np.broadcast(a, b).shape)
    nz = b != 0
    out[nz] = np.abs(a[nz] / b[nz] - 1.0)
    out[~nz & (a != 0)] = np.inf
    return out


def markdown_table(header, rows):
    lines = ["| " + " | ".join(header) + " |", "|" + "---|" * len(header)]
    lines += ["| " + " | ".join(str(c) for c in r) + " |" for r in rows]
    return "\n".join(lines)
