"""Checkpoint and resume of a covariance run over realisations.

Sec. 3.2 estimates covariances from 150 realisations; the running estimate
is the Welford state of the library (FP64: n, mean [d], M2 [d, d], the layout
of ufc_welford_update).  A run that stops after realisation k saves that
state with the index k + 1 of the next realisation and a fingerprint of the
run's configuration; a resumed run loads it and continues the updates from
realisation k + 1.  Because the update is sequential and exact in its order,
resuming in the same order gives the same state bit for bit as an
uninterrupted run; a resumed part kept in its own state and merged
afterwards (ufc_welford_merge, the Chan update) agrees to rounding.

The file is an .npz archive written to a temporary name, flushed to disk and
renamed over the target, so a crash while saving leaves the previous
checkpoint intact.
"""
from __future__ import annotations

import json
import os

import numpy as np

_FORMAT = "ufalcon-welford-1"


def _host_state(state) -> np.ndarray:
    if hasattr(state, "detach"):                     # a torch tensor, host or device
        state = state.detach().cpu().numpy()
    st = np.ascontiguousarray(state)
    if st.dtype != np.float64:
        raise TypeError("a Welford state is float64")
    return st


def save(path: str, state, d: int, next_realisation: int, config: dict | None = None) -> None:
    """Writes the Welford state of a d-dimensional run, the index of the
    next realisation and the run's configuration (a JSON-serialisable dict,
    compared on load) to `path`."""
    st = _host_state(state)
    if st.shape != (1 + d + d * d,):
        raise ValueError(f"state of {st.size} values, expected 1 + d + d^2 = {1 + d + d * d}")
    if next_realisation < 0 or int(st[0]) != st[0] or st[0] > next_realisation:
        raise ValueError("next_realisation must be at least the state's count n")
    cfg = json.dumps(config or {}, sort_keys=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, format=np.array(_FORMAT), state=st, d=np.int64(d),
                 next=np.int64(next_realisation), config=np.array(cfg))
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str, d: int, config: dict | None = None) -> tuple[np.ndarray, int]:
    """(state, next_realisation) of a checkpoint written by save(); raises
    ValueError when the file is of another format, dimension or
    configuration (config None skips the configuration check)."""
    with np.load(path, allow_pickle=False) as z:
        if str(z["format"]) != _FORMAT:
            raise ValueError(f"{path}: not a Welford checkpoint")
        if int(z["d"]) != d:
            raise ValueError(f"{path}: dimension {int(z['d'])}, expected {d}")
        if config is not None and str(z["config"]) != json.dumps(config, sort_keys=True):
            raise ValueError(f"{path}: saved for another configuration")
        st = np.array(z["state"], dtype=np.float64)
        nxt = int(z["next"])
    if st.shape != (1 + d + d * d,):
        raise ValueError(f"{path}: state of {st.size} values")
    return st, nxt
