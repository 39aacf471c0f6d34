"""Shared agent policy evaluated on the sensing plane, written out plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is computed (paper Sec. 3.2)
---------------------------------
One agent per wall grid point (N_CTRLx = Nx, N_CTRLz = Nz), every agent with
the same policy, each observing the portion of the sensing plane above its
actuator and returning one wall-normal velocity.  The policy is the actor of
DDPG (Sec. 3.2), a multilayer perceptron; the paper does not give its
architecture, so the reading here (shared with the library's on-device mode):

* observation of agent (iz, ix): u and v on a periodic wz x wx window centred
  on it, flattened as x[(c wz + dz) wx + dx] = plane[c, (iz + dz - wz//2) mod
  nz, (ix + dx - wx//2) mod nx], c = 0 for u, 1 for v;
* n_hidden (0, 1 or 2) layers h = max(0, W h_prev + b), then one output
  y = W h + b;
* action = u_tau tanh(y) (bounded like the paper's actions, Sec. 3.2) or y.

Weights are a flat vector: per layer W [out][in] row-major, then b [out].
FP64 throughout; the library evaluates the same function in FP32.
"""

from __future__ import annotations

import numpy as np


def layer_shapes(wz: int, wx: int, hidden: tuple) -> list[tuple[int, int]]:
    """(out, in) of every layer, the output layer last."""
    sizes = [2 * wz * wx] + list(hidden) + [1]
    return [(sizes[i + 1], sizes[i]) for i in range(len(sizes) - 1)]


def weight_count(wz: int, wx: int, hidden: tuple) -> int:
    return sum(o * i + o for o, i in layer_shapes(wz, wx, hidden))


def unpack(weights: np.ndarray, wz: int, wx: int, hidden: tuple) -> list[tuple[np.ndarray, np.ndarray]]:
    w = np.asarray(weights, dtype=np.float64).ravel()
    if w.size != weight_count(wz, wx, hidden):
        raise ValueError("weight count does not match the layer sizes")
    out, pos = [], 0
    for o, i in layer_shapes(wz, wx, hidden):
        W = w[pos:pos + o * i].reshape(o, i)
        pos += o * i
        b = w[pos:pos + o]
        pos += o
        out.append((W, b))
    return out


def observations(plane: np.ndarray, wz: int, wx: int) -> np.ndarray:
    """[B][nz][nx][2 wz wx] windows of the sensing plane [B][2][nz][nx]."""
    B, _, nz, nx = plane.shape
    X = np.zeros((B, nz, nx, 2 * wz * wx))
    for iz in range(nz):
        for ix in range(nx):
            k = 0
            for c in range(2):
                for dz in range(wz):
                    for dx in range(wx):
                        X[:, iz, ix, k] = plane[:, c, (iz + dz - wz // 2) % nz, (ix + dx - wx // 2) % nx]
                        k += 1
    return X


def actions(plane: np.ndarray, weights: np.ndarray, wz: int = 1, wx: int = 1, hidden: tuple = (),
            out_tanh: bool = True, u_tau: float = 1.0) -> np.ndarray:
    """Wall action [B][nz][nx] of every agent before the library's clip and
    mean removal."""
    layers = unpack(weights, wz, wx, hidden)
    h = observations(np.asarray(plane, dtype=np.float64), wz, wx)
    for W, b in layers[:-1]:
        h = np.maximum(h @ W.T + b, 0.0)
    W, b = layers[-1]
    y = (h @ W.T + b)[..., 0]
    return u_tau * np.tanh(y) if out_tanh else y
