"""Model, in numpy, of the rounding of the centred array to FP32 that the
batched split-precision path stores (no GPU): why it rounds stochastically.

For float32 data x and an FP64 mean, round-to-nearest of x - mean leaves an
error that is the same for every sample in a binade of |x - mean| and for
either sign of it: an even function of x.  Removing the residual column mean
leaves its correlation with x^2, which biases third moments in proportion to
t, while symmetric data's third moments are of sampling scale 1/sqrt(t): the
relative error grows like sqrt(t).  Stochastic rounding (away from zero with
probability remainder / ulp) makes the error zero-mean and independent of x.
Third moments of the batched workload's data (Student-t(5) mixed, n = 16)
against the exactly centred FP64 data, both sides with their own column mean
removed."""
import numpy as np

import synth


def _m3(Y):
    out = np.empty((Y.shape[1],) * 3)
    for i in range(Y.shape[1]):
        out[i] = (Y[:, i:i + 1] * Y).T @ Y
    return out / Y.shape[0]


def _round_nearest32(v):
    return v.astype(np.float32).astype(np.float64)


def _round_stochastic32(v, u):
    h = v.astype(np.float32)
    over = np.abs(h.astype(np.float64)) > np.abs(v)
    h[over] = np.nextafter(h[over], np.float32(0))                    # toward zero
    up = np.nextafter(h, np.where(v > 0, np.inf, -np.inf).astype(np.float32))
    ulp = np.abs(up.astype(np.float64) - h.astype(np.float64))
    r = np.abs(v - h.astype(np.float64))
    return np.where(u * ulp < r, up, h).astype(np.float64)


def _errors(t):
    X = synth.batch_dataset(t, 16, 12345)
    Xc = X.astype(np.float64) - X.astype(np.float64).mean(0)
    ref = _m3(Xc - Xc.mean(0))
    rn = _round_nearest32(Xc)
    sr = _round_stochastic32(Xc, np.random.default_rng(7).random(Xc.shape))
    rel = lambda Y: np.linalg.norm(_m3(Y - Y.mean(0)) - ref) / np.linalg.norm(ref)
    return rel(rn), rel(sr)


def test_stochastic_rounding_removes_the_growing_bias():
    rn_small, _ = _errors(20000)
    rn_large, sr_large = _errors(175000)
    # round-to-nearest: the relative error grows about like sqrt(t) (x 2.96 here)
    assert rn_large > 2.0 * rn_small, (rn_small, rn_large)
    # stochastic rounding: an order of magnitude below it at the large t
    assert sr_large < rn_large / 4 and sr_large < 1.5e-7, (sr_large, rn_large)
