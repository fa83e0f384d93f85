"""Pins of the oracle's object-inferring loss (Sec. 2.2.1, Eq. 8 with the
regulariser gamma sum |O|^2), CPU only: at the Wiener object it is the
object-eliminated loss of Eq. 12 with zero object gradient and the same dL/da
(the envelope theorem); its gradients match central differences; O = 0 has a
closed form."""

import numpy as np

from oracle import mfbd
from tests import cases


def _case():
    return cases.make_case(n_pix=32, diams=(12.0, 15.0), wavelengths=(6563.0, 8542.0), n_frames=3, n_modes=8,
                           basis="kl", seed=21, weights=[[1.0, 0.5, 1.5], [0.8, 1.2, 1.0]])


def _perturbed(o, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(o.shape) + 1j * rng.standard_normal(o.shape)
    return o + scale * np.abs(o).mean() * d


def test_at_the_wiener_object_it_is_the_eliminated_loss():
    c = _case()
    s, a, d = c["setup"], c["a_eval"][0], c["d"][0]
    l_e, o_w, g_e = mfbd.loss_object_grad_patch(s, a, d)
    l_x, g_x, g_o = mfbd.explicit_loss_grad_patch(s, a, d, o_w)
    assert abs(l_x - l_e) <= 1e-12 * abs(l_e)
    assert np.abs(g_o).max() <= 1e-12 * np.abs(d).max() * np.abs(o_w).max()
    assert np.linalg.norm(g_x - g_e) <= 1e-10 * np.linalg.norm(g_e)


def test_the_wiener_object_is_the_minimum():
    c = _case()
    s, a, d = c["setup"], c["a_eval"][0], c["d"][0]
    l_e, o_w, _ = mfbd.loss_object_grad_patch(s, a, d)
    for seed in range(3):
        l_x, _, _ = mfbd.explicit_loss_grad_patch(s, a, d, _perturbed(o_w, seed))
        assert l_x > l_e


def test_zero_object_closed_form():
    """O = 0: L = sum w |D|^2, g_O = -sum_j w conj(H_j) D_j, dL/da = 0."""
    c = _case()
    s, a, d = c["setup"], c["a_eval"][0], c["d"][0]
    o = np.zeros((2, 32, 32), np.complex128)
    l_x, g_x, g_o = mfbd.explicit_loss_grad_patch(s, a, d, o)
    inter = mfbd.otf_patch(s, a)
    want_l = sum((s.weights[k][:, None, None] * np.abs(d[k]) ** 2).sum() for k in range(2))
    assert abs(l_x - want_l) <= 1e-13 * want_l
    assert not g_x.any()
    for k in range(2):
        want = -(s.weights[k][:, None, None] * inter[k]["H"].conj() * d[k]).sum(axis=0)
        assert np.allclose(g_o[k], want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_coefficient_gradient_central_differences():
    c = _case()
    s, a, d = c["setup"], c["a_eval"][0], c["d"][0]
    _, o_w, _ = mfbd.loss_object_grad_patch(s, a, d)
    o = _perturbed(o_w, 7, 0.2)
    _, g, _ = mfbd.explicit_loss_grad_patch(s, a, d, o)
    h = 2e-4
    fd = np.zeros_like(a)
    for idx in np.ndindex(a.shape):
        vals = []
        for step in (2, 1, -1, -2):
            x = a.copy()
            x[idx] += step * h
            vals.append(mfbd.explicit_loss_grad_patch(s, x, d, o)[0])
        fd[idx] = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
    assert np.linalg.norm(g - fd) <= 3e-7 * np.linalg.norm(g)


def test_object_gradient_central_differences():
    """L is quadratic in O: central differences along Re O(u) and Im O(u)
    give 2 Re g_O(u) and 2 Im g_O(u) to rounding."""
    c = _case()
    s, a, d = c["setup"], c["a_eval"][0], c["d"][0]
    _, o_w, _ = mfbd.loss_object_grad_patch(s, a, d)
    o = _perturbed(o_w, 9, 0.2)
    _, _, g_o = mfbd.explicit_loss_grad_patch(s, a, d, o)
    step = 1e-3 * np.abs(o).mean()
    for k, y, x in ((0, 0, 0), (0, 1, 2), (1, 5, 30), (1, 16, 16), (0, 31, 7)):
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            op, om = o.copy(), o.copy()
            op[k, y, x] += unit * step
            om[k, y, x] -= unit * step
            fd = (mfbd.explicit_loss_grad_patch(s, a, d, op)[0] - mfbd.explicit_loss_grad_patch(s, a, d, om)[0]) / (
                2 * step)
            assert abs(fd - 2 * part(g_o[k, y, x])) <= 1e-6 * (abs(fd) + np.abs(g_o).max() * 1e-3)
