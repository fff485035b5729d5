"""Saturated starting states for the fixed-allele tests: angle indices placed through an
instance's checkpoint."""
import numpy as np


def saturated_start(ng, np_, seed, n_odd, flips, D=100):
    """Angle indices at the bounds (every qubit saturated): rows share one allele pattern
    except n_odd rows with `flips` genes flipped. Returns k[np, ng]."""
    K = D // 4
    rng = np.random.default_rng(seed)
    xs = np.tile(rng.integers(0, 2, ng), (np_, 1))
    for c in rng.choice(np_, n_odd, replace=False):
        xs[c, rng.choice(ng, flips, replace=False)] ^= 1
    return np.where(xs == 1, K, -K).astype(np.int16)


def load_state(inst, k, D=100, byte_state=False):
    """Replaces the angle indices of an instance at generation 0 through its checkpoint (the
    state bytes are the checkpoint's tail: 4n per gene, n = k + K, padded to whole vectors)."""
    K = D // 4
    np_, ng = k.shape
    svec = (ng + 7) // 8
    buf = bytearray(inst.save())
    dt = np.uint8 if byte_state else np.uint16
    nbytes = np_ * svec * 8 * np.dtype(dt).itemsize
    st = np.frombuffer(bytes(buf[-nbytes:]), dtype=dt).reshape(np_, svec * 8).copy()
    st[:, :ng] = (4 * (k.astype(np.int32) + K)).astype(dt)
    buf[-nbytes:] = st.tobytes()
    inst.load(bytes(buf))

