"""Pins of the oracle's masked copies (no GPU): the definition of the
paper's copyFromTargetMasked / copyToTargetMasked (Sec. III.B) -- the
sites whose mask byte is non-zero, in site order -- checked against explicit
loops on small inputs, and the identities a compaction must satisfy."""
import numpy as np
import pytest

import lb_inputs as L
import oracle


def _loop_select(x, mask):
    cols = [x[..., s] for s in range(x.shape[-1]) if mask[s] != 0]
    return np.stack(cols, axis=-1) if cols else np.zeros(x.shape[:-1] + (0,), x.dtype)


@pytest.mark.parametrize("density", [0.0, 0.03, 0.5, 1.0])
def test_select_matches_loop(density):
    n = 257
    mask = (L.uniform(800, n, 0, 1) < density).astype(np.uint8) * np.uint8(1 + L.uniform_int(801, 1, 0, 200)[0])
    x = L.uniform(802, 19 * n, -1, 1).reshape(19, n)
    got = oracle.select_sites(x, mask)
    assert got.shape == (19, int((mask != 0).sum()))
    assert np.array_equal(got, _loop_select(x, mask))


def test_scatter_inverts_select():
    n = 300
    mask = (L.uniform(803, n, 0, 1) < 0.2).astype(np.uint8)
    x = L.uniform(804, 3 * n, -1, 1).reshape(3, n)
    y = L.uniform(805, 3 * n, -1, 1).reshape(3, n)
    z = oracle.scatter_sites(y, mask, oracle.select_sites(x, mask))
    keep = mask != 0
    assert np.array_equal(z[:, keep], x[:, keep]) and np.array_equal(z[:, ~keep], y[:, ~keep])
    # loop form of the scatter
    w = y.copy()
    k = 0
    for s in range(n):
        if mask[s]:
            w[:, s] = x[:, s]
            k += 1
    assert np.array_equal(z, w) and k == keep.sum()
