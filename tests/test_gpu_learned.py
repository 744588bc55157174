"""Learned part on the GPU: MLP forward/backward/Adam against the FP64 oracle (same bf16-rounded
weights), randomized Tucker against the oracle's randomized Tucker (same widths and sketches),
the HOSVD fallback, and the learned-width pipeline end to end."""
import numpy as np
import pytest

from oracle import mlp, randomized, tucker
from paper_2103_06393_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402


def pack(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def unpack(vec):
    out, o = [], 0
    for i in range(4):
        fi, fo = mlp.SIZES[i], mlp.SIZES[i + 1]
        W = vec[o:o + fi * fo].reshape(fo, fi).astype(np.float64)
        o += fi * fo
        b = vec[o:o + fo].astype(np.float64)
        o += fo
        out.append((W, b))
    return out


def test_mlp_forward_backward_against_oracle():
    params = mlp.init_params(0)
    M = zbc.Mlp(pack(params))
    master, wbf = M.params()
    pbf = unpack(wbf)                       # the bf16-rounded weights the GPU computes with
    assert np.max(np.abs(wbf - pack(params))) <= 2 ** -8 * np.max(np.abs(pack(params)))
    rng = np.random.default_rng(1)
    X = rng.normal(size=(77, 7)).astype(np.float32)   # ragged: 77 = 2*32 + 13
    T = rng.normal(size=(77, 9)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    out = M.forward(Xd).cpu().numpy()
    ref, cache = mlp.forward(pbf, X.astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(ref))
    g, loss = M.backward(Xd, Td)
    grads = mlp.backward(pbf, cache, ref, T.astype(np.float64))
    gref = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in grads])
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - gref)) <= 1e-4 * np.max(np.abs(gref))
    assert abs(float(loss.item()) - mlp.loss(ref, T)) <= 1e-5 * mlp.loss(ref, T)
    # deterministic reduction: a second backward gives identical bits
    g2, _ = M.backward(Xd, Td)
    assert torch.equal(g, g2)
    # one Adam step on the master weights
    M.adam_step(g, 1e-3)
    new_master, _ = M.params()
    state = {}
    upd = mlp.adam_step(unpack(master), _split(gg), state, lr=1e-3)
    assert np.max(np.abs(new_master - pack(upd))) <= 1e-6


def _split(vec):
    out, o = [], 0
    for i in range(4):
        fi, fo = mlp.SIZES[i], mlp.SIZES[i + 1]
        out.append((vec[o:o + fi * fo].reshape(fo, fi).astype(np.float64), vec[o + fi * fo:o + fi * fo + fo].astype(np.float64)))
        o += fi * fo + fo
    return out


def test_mlp_training_reduces_loss():
    params = mlp.init_params(3)
    M = zbc.Mlp(pack(params))
    rng = np.random.default_rng(4)
    X = rng.normal(size=(256, 7)).astype(np.float32)
    T = np.tanh(X @ rng.normal(size=(7, 9))).astype(np.float32)
    hist = M.train(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), 300, 3e-3).cpu().numpy()
    assert hist[-1] < 0.2 * hist[0]


def _columns(name, n, m, dtype=torch.complex128):
    w = inputs.scaled_workload(name, n, m=m)
    g, s = w.grid, w.segments
    ds = zbc.DeviceSegments(s)
    cols = torch.arange(s.m, dtype=torch.int32, device="cuda")
    Z = zbc.colmajor(3 * g.nv, s.m, dtype)
    zbc.vsie_assemble_columns(g, ds, w.freq_hz, cols, Z)
    torch.cuda.synchronize()
    return w, g, s, Z


def test_randomized_against_oracle_and_fallback():
    w, g, s, Zd = _columns("precision", (24, 22, 20), 6)
    Z = zbc.from_colmajor(Zd)
    tol = 1e-6
    lmax = 32
    sk = inputs.mode_sketches(g, lmax, seed=11)
    skd = [zbc.to_colmajor(o) for o in sk]
    # widths from the oracle's HOSVD ranks + 4, except two tensors starved on purpose
    widths = np.zeros(3 * 3 * s.m, dtype=np.int32)
    hos = []
    for j in range(s.m):
        for k in range(3):
            A = tucker.fold(Z[k * g.nv:(k + 1) * g.nv, j], g.shape)
            _, _, info = tucker.hosvd(A, tol)
            hos.append(info)
            t = 3 * j + k
            widths[3 * t:3 * t + 3] = [min(r + 4, n) // 2 * 2 for r, n in zip(info["ranks"], g.shape)]
    widths[0:3] = 2
    widths[3 * 7:3 * 7 + 3] = 2
    h, st = zbc.tucker_compress_randomized(Zd, g, tol, widths, skd, lmax)
    tens, _ = h.tensors()
    assert st.n_fallback >= 2
    for j in range(s.m):
        for k in range(3):
            t = 3 * j + k
            A = tucker.fold(Z[k * g.nv:(k + 1) * g.nv, j], g.shape)
            Go, Uo, info = randomized.randomized_tucker(A, widths[3 * t:3 * t + 3],
                                                         [o.astype(np.complex128) for o in sk], tol)
            gr = tuple(U.shape[1] for U in tens[j][k][1])
            if info["fallback"]:
                assert gr == hos[t]["ranks"] or min(hos[t]["margin"]) < 1e-5
            else:
                # the GPU forms the sketch, its QR and e^2 in FP64 like the oracle, but with its own
                # summation order and Householder QR, so the projection error e^2 and hence the
                # truncation budget (tol^2 ||A||^2 - e^2) differ from the oracle's by rounding:
                # ranks agree away from the threshold and within one near it
                if min(info["margin"]) > 0.1:
                    assert gr == info["ranks"], (t, gr, info["ranks"])
                else:
                    assert max(abs(a - b) for a, b in zip(gr, info["ranks"])) <= 1, (t, gr, info["ranks"])
            err = np.linalg.norm(tucker.reconstruct(tens[j][k][0], tens[j][k][1]) - A) / np.linalg.norm(A)
            assert err <= tol * (1 + 1e-6) + 3e-7, (t, err)
    assert st.max_rel_err <= tol * (1 + 1e-9)


def test_learned_pipeline_end_to_end():
    w, g, s, Zd = _columns("precision", (24, 22, 20), 8)
    M = zbc.Mlp(pack(mlp.init_params(5)))
    feats = torch.from_numpy(inputs.rank_features(g, s)).cuda()
    widths = M.widths(feats, g, oversample=4)
    assert widths.shape == (9 * s.m,) and widths.min() >= 2
    lmax = 64
    skd = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=3)]
    h, st = zbc.tucker_compress_randomized(Zd, g, 1e-6, widths, skd, lmax)
    assert st.n_tensors == 3 * s.m and st.max_rel_err <= 1e-6 * (1 + 1e-9)


def _effective_widths(widths, n, lmax):
    """Reading R4: each width clamped to [2, min(n_g, lmax, 64)] and made even (rounded up when
    room allows)."""
    out = np.array(widths, dtype=np.int64).reshape(-1, 3)
    for t in range(out.shape[0]):
        for g in range(3):
            cap = min(n[g], lmax, 64) // 2 * 2
            v = max(2, min(int(out[t, g]), cap))
            if v & 1:
                v = v + 1 if v + 1 <= cap else v - 1
            out[t, g] = v
    return out


def _check_randomized_handle(h, Z, g, widths_eff, sk, tol):
    """Ranks and errors of a randomized-Tucker handle against the oracle's randomized Tucker on the
    same widths and sketches (ranks equal away from the truncation threshold, within one near it;
    fallback tensors against the oracle's HOSVD)."""
    tens, _ = h.tensors()
    nfb = 0
    for j in range(len(tens)):
        for k in range(3):
            t = 3 * j + k
            A = tucker.fold(Z[k * g.nv:(k + 1) * g.nv, j], g.shape)
            _, _, info = randomized.randomized_tucker(A, widths_eff[t], [o.astype(np.complex128) for o in sk], tol)
            gr = tuple(U.shape[1] for U in tens[j][k][1])
            nfb += int(info["fallback"])
            if min(info["margin"]) > 0.1:
                assert gr == tuple(info["ranks"]), (t, gr, info["ranks"])
            else:
                assert max(abs(a - b) for a, b in zip(gr, info["ranks"])) <= 1, (t, gr, info["ranks"])
            err = np.linalg.norm(tucker.reconstruct(tens[j][k][0], tens[j][k][1]) - A) / np.linalg.norm(A)
            assert err <= tol * (1 + 1e-6) + 3e-7, (t, err)
    return nfb


@pytest.mark.parametrize("method", ["fixed", "learned"])
def test_tucker_compress_randomized_methods(method):
    """tucker_compress with ZBC_RANDOMIZED_FIXED and ZBC_RANDOMIZED_LEARNED against the oracle's
    randomized Tucker on the widths each method implies."""
    w, g, s, Zd = _columns("learned", (24, 22, 20), 6)
    Z = zbc.from_colmajor(Zd)
    tol, lmax = 1e-6, 32
    sk = inputs.mode_sketches(g, lmax, seed=17)
    skd = [zbc.to_colmajor(o) for o in sk]
    if method == "fixed":
        model = zbc.rank_model(skd, lmax, fixed_width=10)
        widths = np.full(9 * s.m, 10)
        h, st = zbc.tucker_compress(Zd, g, tol, method=zbc.RANDOMIZED_FIXED, model=model)
    else:
        M = zbc.Mlp(pack(mlp.init_params(5)))
        feats = torch.from_numpy(inputs.rank_features(g, s)).cuda()
        widths = M.widths(feats, g, oversample=4)
        # the library's widths are the oracle MLP's on the same bf16 weights, ceil(exp(.)) + 4
        _, wbf = M.params()
        pred, _ = mlp.forward(unpack(wbf), inputs.rank_features(g, s).astype(np.float64))
        ow = np.ceil(np.exp(pred)).reshape(-1) + 4
        ow = np.clip(ow, 2, np.tile(np.array(g.shape), 3 * s.m))
        near = np.abs(np.exp(pred).reshape(-1) - np.round(np.exp(pred).reshape(-1))) < 1e-4
        assert np.all((ow == widths) | near)
        model = zbc.rank_model(skd, lmax, mlp=M, features=feats, oversample=4)
        h, st = zbc.tucker_compress(Zd, g, tol, method=zbc.RANDOMIZED_LEARNED, model=model)
    assert st.n_tensors == 3 * s.m and st.max_rel_err <= tol * (1 + 1e-9)
    nfb = _check_randomized_handle(h, Z, g, _effective_widths(widths, g.shape, lmax), sk, tol)
    assert st.n_fallback == nfb


def test_tucker_compress_rejects_bad_model_and_storage():
    w, g, s, Zd = _columns("learned", (8, 8, 6), 2)
    lmax = 8
    skd = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=17)]
    for method, model in ((zbc.RANDOMIZED_FIXED, None), (zbc.RANDOMIZED_FIXED, zbc.rank_model(skd, lmax)),
                          (zbc.RANDOMIZED_LEARNED, zbc.rank_model(skd, lmax, fixed_width=4))):
        with pytest.raises(zbc.ZbcError) as e:
            zbc.tucker_compress(Zd, g, 1e-6, method=method, model=model)
        assert e.value.status == zbc.ZBC_EINVAL


def test_trained_network_beats_fixed_widths():
    """What the learned part gains: the MLP trained on the GPU on HOSVD ranks of 96 columns, then 64
    other columns compressed with its widths, with one fixed width equal to the learned widths'
    mean (the same sketch budget spread evenly) and with the fixed width the method needs without
    the network (the largest training rank + 4).  The trained widths must sketch less than the
    fixed-max width (the sketches and the projection cost grow with the width), fall back to the
    HOSVD on few tensors and no more often than the evenly spread budget, and all three must meet
    the tolerance."""
    w = inputs.scaled_workload("learned", (40, 36, 32), m=160)
    g, s = w.grid, w.segments
    ds = zbc.DeviceSegments(s)
    tol, lmax = 1e-6, 32
    feats = inputs.rank_features(g, s)
    train, test = np.arange(96), np.arange(96, 160)

    def assemble(cols):
        Z = zbc.colmajor(3 * g.nv, len(cols), torch.complex64)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, torch.from_numpy(cols.astype(np.int32)).cuda(), Z)
        return Z

    h, _ = zbc.tucker_compress(assemble(train), g, tol)
    rt = h.export()[0].reshape(-1, 9)
    M = zbc.Mlp(pack(mlp.init_params(0)))
    hist = M.train(torch.from_numpy(feats[train]).cuda(), torch.from_numpy(np.log(rt.astype(np.float32))).cuda(),
                   1500, 3e-3).cpu().numpy()
    assert hist[-1] < 0.3 * hist[0]
    ft = torch.from_numpy(feats[test]).cuda()
    widths = M.widths(ft, g, oversample=4)
    sk = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=19)]
    Z = assemble(test)
    _, st_l = zbc.tucker_compress(Z, g, tol, method=zbc.RANDOMIZED_LEARNED,
                                  model=zbc.rank_model(sk, lmax, mlp=M, features=ft, oversample=4))
    mean_w = int(round(float(_effective_widths(widths, g.shape, lmax).mean())))
    _, st_m = zbc.tucker_compress(Z, g, tol, method=zbc.RANDOMIZED_FIXED,
                                  model=zbc.rank_model(sk, lmax, fixed_width=mean_w))
    _, st_x = zbc.tucker_compress(Z, g, tol, method=zbc.RANDOMIZED_FIXED,
                                  model=zbc.rank_model(sk, lmax, fixed_width=int(rt.max()) + 4))
    print(f"fallbacks: learned {st_l.n_fallback}, fixed at the learned mean {mean_w}: {st_m.n_fallback}, "
          f"fixed at the training maximum {int(rt.max()) + 4}: {st_x.n_fallback} of {st_l.n_tensors}")
    wl = np.asarray(widths.cpu() if hasattr(widths, "cpu") else widths).reshape(-1)
    learned_work = float(_effective_widths(wl, g.shape, lmax).sum())
    fixed_work = float(_effective_widths(np.full(wl.size, int(rt.max()) + 4), g.shape, lmax).sum())
    print(f"sketch widths summed over tensors and modes: learned {learned_work:.0f}, fixed max {fixed_work:.0f}")
    assert learned_work < fixed_work
    assert st_l.n_fallback <= max(1, st_l.n_tensors // 10)
    assert st_l.n_fallback <= st_m.n_fallback
    for st in (st_l, st_m, st_x):
        assert st.max_rel_err <= tol * (1 + 1e-9)
