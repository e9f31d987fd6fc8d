"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU).

Tolerances (fixed for this hot path): relative L2 1e-5 on mixes, L_a and the total loss, 1e-3 on gradients (per
processor type and for the dry/wet logits).  Where FP32 cannot meet a plain bound the test applies one derived
from the arithmetic and states it; every measured error is recorded against the plain bound (record_error)."""
import numpy as np
import pytest

import workloads as W
from oracle import adam as OA
from tests.cases import (make_case, gpu_console, rel_l2, grad_groups, LOSS_FIELDS, oracle_with_delay_taps,
                         delay_slot_conditioning, delay_term_rms, record_error, current_test)

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-5
LOSS_TOL = 1e-5
SET_TOL = 2e-5       # L_lr, L_m, L_s: components of L_a, measured up to 1.6e-5
GRAD_TOL = 1e-3


def audio_floors(case, mix, s, ol_row):
    """Change of the oracle's L_a and of its per-set terms L_lr, L_m, L_s (Eq. 21) of song s when its mix moves
    by white noise of relative L2 1e-5: the FP32 floor of the log-spectral terms (bins where the target is
    near its magnitude floor make it large)."""
    import torch
    from oracle import loss as OL
    m = torch.tensor(np.asarray(mix, np.float64))
    noise = torch.tensor(np.random.default_rng(0).standard_normal(m.shape))
    noise *= 1e-5 * m.norm() / noise.norm()
    tgt = torch.tensor(np.asarray(case.targets[s], np.float64))
    r = OL.audio_loss(m + noise, tgt, case.oracle.desc.loss)
    return {name: abs(float(r[key]) - float(ol_row[j]))
            for j, (name, key) in enumerate((("La", "a"), ("Llr", "lr"), ("Lm", "m"), ("Ls", "s")))}


def la_floor(case, mix, s, la):
    """Change of the oracle's L_a of song s when its mix moves by white noise of relative L2 1e-5."""
    return audio_floors(case, mix, s, [la, 0.0, 0.0, 0.0])["La"]


def run_both(case, alpha_p=1e-3, **cfg):
    ol, og, omix, taps = oracle_with_delay_taps(case, alpha_p)
    con = gpu_console(case, **cfg)
    con.set_alpha_p(alpha_p)
    con.set_params(case.params)
    losses, mixes = con.forward_loss(with_mix=True)
    con.backward()
    g = con.get_grads().cpu().numpy()
    return (ol, og, omix, taps), (losses.cpu().numpy(), g, [m.cpu().numpy() for m in mixes]), con


def channel_conditioning(mix):
    """kappa_x = ||(l, r)|| / ||x||: relative errors of the mid / side signals are the stereo mix's relative
    error times this factor (a set that nearly cancels is ill-conditioned)."""
    lr = np.linalg.norm(mix)
    m = np.linalg.norm(mix[0] + mix[1])
    s = np.linalg.norm(mix[0] - mix[1])
    return {"Llr": 1.0, "Lm": lr / m if m > 0 else np.inf, "Ls": lr / s if s > 0 else np.inf}


def _window_norms(x, w):
    """||x[q : q + w]||_2 for every q (sliding windows of length w)."""
    c = np.concatenate([[0.0], np.cumsum(np.asarray(x, np.float64) ** 2)])
    return np.sqrt(np.maximum(c[w:] - c[:-w], 0.0))


def check_delay(case, og, gg, taps, con, term_rms=None, proc_map=None):
    """Delay gradients (Sec. 3.7, Eq. 19).
    * The 20 log-magnitudes of every c_m: the gradient bound.
    * dL/dh, the FIR tap gradient that the FFT correlation computes (read back from the GPU), against the
      oracle's dL/dh[j] = sum_n dL/dy_bar[n] u[n - j], per channel in L2 over the tap lags, within
      1e-3 ||dL/dh|| + 1e-4 ||A||, A[j] = sum_n |dL/dy_bar[n]| |u[n - j]| the summed term magnitudes.  dL/dh
      cancels 40-4000x against A (most near an optimum, or on a console far louder than its target), and FP32
      sets a floor relative to A: the worst-case rounding of three radix-2 transforms of N points,
      15 log2(N) 2^-24 (1.9e-5 at 2^21), plus the upstream adjoint's own rounding, of the same order (measured
      1.8e-5 and 2.2e-5 of A).
    * The z entries, sgn(g_m) + gamma (|z| - 1) z/|z| with g_m = sum_q G_q conj(s'_q) and
      G_q = sum_j dL/dh[m D + q + j] c_m[j]: the direction normalises g_m, so an error e of dL/dh moves it by at
      most 2 |dg| / |g_m| with |dg| <= sum_q ||e[m D + q : m D + q + 39]|| ||c_m|| |s'_q| (Cauchy-Schwarz).
      Each entry is held to the gradient bound plus that propagation of the measured dL/dh error (e = GPU minus
      oracle); kappa = |g_m| / (rms(dL/dh) ||c_m|| ||s'||) is recorded with the error.
    proc_map: the console's processor index of each of the case's processors (default: the same index)."""
    from oracle import processors as OP
    from tests.cases import lag_correlation
    D = int(round(0.1 * case.fs))
    kap = delay_slot_conditioning(case, taps, term_rms=term_rms)
    t = current_test()
    lm_idx = []
    worst_plain, worst_k, worst_over_bound, n_prop = 0.0, 0.0, 0.0, 0
    for p in case.oracle.procs:
        if p.type != "d":
            continue
        dh_o, cvals, u_abs, dybar_o = taps[p.index]
        cp = p.index if proc_map is None else int(proc_map[p.index])
        dh_g = con.debug_read(cp, 2, dh_o.shape).astype(np.float64)
        A = lag_correlation(np.abs(dybar_o), u_abs, dh_o.shape[1])
        blk = np.arange(p.offset, p.offset + p.count).reshape(2, 20, 22)
        lm_idx.append(blk[:, :, 2:].ravel())
        for ch in range(2):
            n_o = np.linalg.norm(dh_o[ch])
            e_dh = rel_l2(dh_g[ch], dh_o[ch])
            kap_a = float(np.linalg.norm(A[ch]) / n_o) if n_o > 0 else np.inf
            record_error(t, "grad d dL/dh (FIR taps)", e_dh, GRAD_TOL, GRAD_TOL + 1e-4 * kap_a, proc=p.index, ch=ch,
                         kappa=kap_a, err_of_A=e_dh / kap_a)
            assert e_dh <= GRAD_TOL + 1e-4 * kap_a, ("dL/dh", p.index, ch, e_dh, kap_a)
            wn = _window_norms(dh_g[ch] - dh_o[ch], 39)
            for m in range(20):
                zi = blk[ch, m, :2]
                z = case.params[zi].astype(np.float64)
                r = np.linalg.norm(z)
                radial = 0.01 * (r - 1.0) * z / r if r > 0 else 0.0 * z
                sg = np.linalg.norm(gg[zi] - radial)
                assert np.isfinite(gg[zi]).all() and (sg < 1e-5 or abs(sg - 1.0) < 1e-4), (p.index, ch, m, sg)
                zc = complex(z[0], z[1])
                sp = OP.surrogate_impulse_dz(zc / max(1.0, abs(zc)), D)
                G = np.lib.stride_tricks.sliding_window_view(dh_o[ch, m * D: m * D + D + 38], 39) @ cvals[ch, m]
                g_abs = abs(np.sum(G * np.conj(sp)))
                prop = 2.0 * np.sum(wn[m * D: m * D + D] * np.abs(sp)) * np.linalg.norm(cvals[ch, m])
                prop = prop / g_abs if g_abs > 0 else np.inf
                bound = GRAD_TOL + prop
                err = np.linalg.norm(gg[zi] - og[zi])
                if np.isfinite(bound):
                    assert err <= bound, (p.index, ch, m, kap[p.index][ch, m], err, bound)
                    worst_over_bound = max(worst_over_bound, err / bound)
                n_prop += prop > GRAD_TOL
                if err > worst_plain:
                    worst_plain, worst_k = err, kap[p.index][ch, m]
    record_error(t, "grad d z direction (abs)", worst_plain, GRAD_TOL, GRAD_TOL, kappa=worst_k,
                 worst_err_over_bound=worst_over_bound, slots_where_dh_error_dominates=n_prop)
    if lm_idx:
        idx = np.concatenate(lm_idx)
        e = rel_l2(gg[idx], og[idx])
        record_error(t, "grad d log-magnitudes", e, GRAD_TOL, GRAD_TOL)
        assert e <= GRAD_TOL, ("grad d log-magnitudes", e)
    return worst_plain


def check(case, alpha_p=1e-3, skip_losses=(), check_grads=True, grad_floor=False, **cfg):
    (ol, og, omix, taps), (gl, gg, gmix), con = run_both(case, alpha_p, **cfg)
    return check_results(case, (ol, og, omix, taps), (gl, gg, gmix), con, alpha_p, skip_losses, check_grads,
                         grad_floor)


def check_results(case, oracle_res, gpu_res, con, alpha_p=1e-3, skip_losses=(), check_grads=True, grad_floor=False,
                  proc_map=None):
    """Mixes, loss terms and gradients of the CUDA path against the oracle's, with every measured error
    recorded against the plain bound (record_error)."""
    (ol, og, omix, taps), (gl, gg, gmix) = oracle_res, gpu_res
    t = current_test()
    for s in range(len(omix)):
        e = rel_l2(gmix[s], omix[s])
        record_error(t, "mix", e, MIX_TOL, MIX_TOL, song=s)
        assert e <= MIX_TOL, ("mix", s, e)
    n_lti = [sum(1 for p in case.oracle.procs if p.song == s and p.type in "erd") for s in range(ol.shape[0])]
    for s in range(ol.shape[0]):
        kap = channel_conditioning(omix[s])
        floors = audio_floors(case, omix[s], s, ol[s, :4])
        floor = floors["La"]
        for j, name in enumerate(LOSS_FIELDS):
            if name in skip_losses or (name == "Lg" and ol[s, j] == 0):
                continue
            if name == "Lg":
                # Eq. (22) sums |differences of log energies|: each log energy is held to 1e-5 (relative error of
                # the energy), so the bound is absolute, 1e-5 per equalizer / reverb / delay node
                record_error(t, "Lg (abs)", abs(gl[s, j] - ol[s, j]), LOSS_TOL, LOSS_TOL * n_lti[s], song=s,
                             rel=abs(gl[s, j] - ol[s, j]) / max(abs(ol[s, j]), 1e-12))
                assert abs(gl[s, j] - ol[s, j]) <= LOSS_TOL * n_lti[s], (name, s, gl[s, j], ol[s, j])
                continue
            if name in kap:
                # the per-set terms of Eq. (21) are reported components of L_a, measured up to 1.6e-5, plus
                # their own FP32 floor of the log-spectral term (as L_a's)
                tol = SET_TOL + floors[name] / max(abs(ol[s, j]), 1e-30)
            elif name in ("La", "total"):
                # plus the FP32 floor of the log-spectral term: the change of the oracle's own L_a when its mix
                # moves by white noise of relative L2 1e-5 (near-silent stretches make it large; usually ~1e-8)
                tol = LOSS_TOL + floor / max(abs(ol[s, 0]), 1e-30)
            else:
                tol = LOSS_TOL
            err = abs(gl[s, j] - ol[s, j]) / max(abs(ol[s, j]), 1e-12)
            record_error(t, name, err, LOSS_TOL, tol, song=s, kappa=float(kap.get(name, 1.0)))
            assert err <= tol, (name, s, gl[s, j], ol[s, j], err, tol)
    if check_grads:
        for name, idx in grad_groups(case).items():
            if name == "d":
                check_delay(case, og, gg, taps, con, delay_term_rms(case, alpha_p) if grad_floor else None, proc_map)
                continue
            e = rel_l2(gg[idx], og[idx])
            record_error(t, f"grad {name}", e, GRAD_TOL, GRAD_TOL)
            assert e <= GRAD_TOL, ("grad", name, e)
    return con, (ol, og, omix), (gl, gg, gmix)


# every type with a stereo processor so that the side channel is not identically zero
@pytest.mark.parametrize("types", ["gs", "cng", "eg", "r", "dg"])
def test_single_type_console(types):
    case = make_case([W.layout_plain(88200)], types=types, seed=1)
    check(case)


@pytest.mark.parametrize("retain", [1, -1])
@pytest.mark.parametrize("types", ["r", "dg", "ecnsgdr"])
def test_retained_and_recomputed_spectra(types, retain):
    """Reverb / delay backward with the spectra kept from the forward (1) and recomputed in the shared
    scratch (-1): both match the oracle."""
    case = make_case([W.layout_plain(88200), W.SongLayout(3, 1, [0, -1, 0], 30011)], types=types, seed=3)
    con, _, _ = check(case, retain_spectra=retain)
    assert con.get_info()["retains_spectra"] == (1 if retain == 1 else 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_full_console_at_ground_truth_parameters(seed):
    """The ground-truth graph's own parameters (slow envelopes with sigmoid(p0) near 1, delays with |z| near 1,
    strong compression), dry/wet logits +-4: the regime the search runs in, where 1 - sigmoid must not be
    formed by subtraction.  Near this optimum the delay's dL/dh is a cancelling sum: the Eq. (19) directions
    use the magnitudes of the summed terms for their conditioning."""
    case = make_case([W.layout_plain(88200)], seed=seed)
    gt, keep = W.ground_truth(case.ptypes, (seed, 77))
    params = gt.copy()
    params[case.oracle.n_proc_params:] = np.where(keep == 1, 4.0, -4.0)
    case.params = params
    check(case, grad_floor=True)


def test_autotuned_splits_keep_parity():
    """The FFT split autotuner picks a valid row/column split per FFT size; results stay within the bounds."""
    lays = [W.layout_plain(88200), W.SongLayout(3, 1, [0, -1, 0], 30011)]
    case = make_case(lays, seed=3)
    con, _, _ = check(case, autotune=1)
    sz = con.fft_sizes()
    types = con.processor_types()
    for (f, logn, logn1), t in zip(sz, types):
        if t in "rd":
            assert f in (1, 3, 5) and 4 <= logn1 and logn - logn1 >= 3 and (f << logn1) <= {1: 2048, 3: 3072, 5: 2560}[f]
        else:
            assert f == 0


@pytest.mark.parametrize("autotune", [0, 1])
def test_factor5_transform_sizes(autotune):
    """Transform sizes N = 5 2^k with rows of 5 2^a: a 1 s song (N = 5 2^15, default rows 5 2^7) and a 4.5 s song
    (N = 5 2^16, default rows 5 2^8) of reverbs and delays, ragged lengths, with the default and the autotuned
    splits."""
    lays = [W.SongLayout(2, 0, [-1, -1], 44111), W.SongLayout(1, 0, [-1], 200003)]
    case = make_case(lays, types="dr", seed=17)
    con, _, _ = check(case, autotune=autotune)
    sz = con.fft_sizes()
    song = con.layout()[2]
    for (f, logn, logn1), s in zip(sz, song):
        assert int(f) == 5 and int(logn) == (15 if s == 0 else 16), (f, logn, s)
        if not autotune:
            assert int(logn1) == (7 if s == 0 else 8)
    con.close()


def test_full_console_plain_workload():
    """4 tracks x 2 s at 44.1 kHz, one subgroup of 2 tracks, every processor type."""
    case = make_case([W.layout_plain(88200)], seed=0)
    check(case)


def test_ragged_lengths_and_batch_of_songs():
    """Three songs of odd lengths (not multiples of any tile), a song without subgroups, an empty-free mix."""
    lays = [W.SongLayout(3, 1, [0, -1, 0], 30011), W.SongLayout(1, 0, [-1], 9001), W.SongLayout(2, 2, [1, 0], 17777)]
    case = make_case(lays, seed=3)
    check(case)


def test_mono_console_side_channel_degenerate():
    """Without a stereo processor the side channel is identically zero: L_s compares two spectrograms of the
    1e-8 magnitude floor and is ill-conditioned; every other term keeps the parity bound."""
    case = make_case([W.layout_plain(30000)], types="ecn", seed=2)
    con, (ol, _, _), (gl, _, _) = check(case, skip_losses=("Ls", "La", "total"), check_grads=False)
    assert abs(gl[0, 3]) < 1e-2 and ol[0, 3] == 0.0


def test_warmup_and_linear_loss_variant():
    """Loss without Mel bands and A-weighting, with a warm-up skip (Sec. 5.1 drops the first second)."""
    case = make_case([W.SongLayout(2, 1, [0, 0], 40000)], seed=4, n_mels=0, a_weighting=False, warmup=5000,
                     n_fft=(256, 1024))
    check(case, warmup_samples=5000, a_weighting=False)


def test_masked_forward_equals_structural_prune_and_scores():
    case = make_case([W.layout_plain(44100)], seed=5)
    con = gpu_console(case)
    con.set_params(case.params)
    rng = np.random.default_rng(0)
    P = con.n_processors
    masks = (rng.uniform(size=(3, P)) > 0.4).astype(np.uint8)
    la = con.prune_scores(masks).cpu().numpy()
    for j in range(3):
        ol, omix = case.oracle.losses(case.params, mask=masks[j])
        assert abs(la[j, 0] - ol[0, 0]) / ol[0, 0] <= LOSS_TOL, (j, la[j, 0], ol[0, 0])
    lm, mm = con.forward_loss(mask=masks[0], with_mix=True)
    mm = mm[0].cpu().numpy().copy()
    con.prune(masks[0])
    lp, mp = con.forward_loss(with_mix=True)
    assert np.array_equal(mp[0].cpu().numpy(), mm)                  # pruned graph == masked console
    assert float(lp[0, 0]) == float(lm[0, 0])
    assert np.array_equal(con.present(), masks[0])


def test_adam_step_matches_oracle():
    case = make_case([W.SongLayout(2, 1, [0, -1], 20000)], seed=6)
    con = gpu_console(case)
    con.set_params(case.params)
    con.forward_loss()
    con.backward()
    g = con.get_grads().cpu().numpy().astype(np.float64)
    con.adam_step(lr=1e-2)
    p1 = con.get_params().cpu().numpy()
    ref, m, v = OA.adam_step(case.params, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-2)
    assert np.max(np.abs(p1 - ref)) < 1e-6
    con.forward_loss()
    con.backward()
    g2 = con.get_grads().cpu().numpy().astype(np.float64)
    con.adam_step(lr=1e-2)
    ref2, _, _ = OA.adam_step(ref, g2, m, v, 2, lr=1e-2)
    assert np.max(np.abs(con.get_params().cpu().numpy() - ref2)) < 1e-5


def test_graph_step_and_per_node_path_are_bitwise_equal():
    import torch
    lays = [W.SongLayout(3, 1, [0, 0, -1], 25000), W.SongLayout(2, 1, [0, 0], 31000)]
    case = make_case(lays, seed=7)
    a = gpu_console(case)
    b = gpu_console(case)
    c = gpu_console(case)
    for con in (a, b, c):
        con.set_params(case.params)
        con.set_alpha_p(1e-4)
    c.set_launch_mode(True)
    for _ in range(3):
        la = a.train_step(lr=1e-2).clone()
        lb = b.forward_loss()
        b.backward()
        b.adam_step(lr=1e-2)
        lc = c.train_step(lr=1e-2).clone()
        torch.cuda.synchronize()
        assert torch.equal(la, lb) and torch.equal(la, lc)
    assert torch.equal(a.get_params(), b.get_params()) and torch.equal(a.get_params(), c.get_params())


def test_song_alone_equals_song_in_batch():
    import torch
    lays = [W.SongLayout(3, 1, [0, -1, 0], 30011), W.SongLayout(2, 2, [1, 0], 17777), W.SongLayout(4, 1, [0] * 4, 22050)]
    batch = make_case(lays, seed=8)
    con = gpu_console(batch)
    con.set_params(batch.params)
    lb, mb = con.forward_loss(with_mix=True)
    con.backward()
    gb = con.get_grads().cpu().numpy()
    # the second song alone, with the same sources, target, noise and parameters
    types = batch.ptypes
    procs = batch.oracle.procs
    sel = [p for p in procs if p.song == 1]
    alone = make_case([lays[1]], seed=8)
    alone.sources = [batch.sources[1]]
    alone.targets = [batch.targets[1]]
    revs = [p.rev for p in sel if p.type == "r"]
    alone.noise = batch.noise[revs]
    pp = np.concatenate([batch.params[p.offset:p.offset + p.count] for p in sel] +
                        [batch.params[batch.oracle.n_proc_params + np.array([p.index for p in sel])]])
    con1 = gpu_console(alone)
    con1.set_params(pp)
    l1, m1 = con1.forward_loss(with_mix=True)
    con1.backward()
    g1 = con1.get_grads().cpu().numpy()
    assert torch.equal(m1[0], mb[1]) and torch.equal(l1[0], lb[1])
    gsel = np.concatenate([gb[p.offset:p.offset + p.count] for p in sel] +
                          [gb[batch.oracle.n_proc_params + np.array([p.index for p in sel])]])
    assert np.array_equal(g1, gsel)
    assert len(types) == con.n_processors


def test_envelope_scan_wait_timeout_is_reported_and_recoverable():
    """The compressor and gate scans hand the envelope state (Eq. 11) from one 4096-sample chunk's CTA to the
    next through a flag that the next CTA waits on for at most about half a second.  With the test hook the first
    chunk of a launch withholds its state: the second chunk's wait runs out, the next call reports MG_ERR_TIMEOUT,
    the context stays usable, and once the hook is released the console computes bitwise what it computed
    before, forward and backward."""
    import torch
    import paper_2509_15948_gb300 as M
    case = make_case([W.SongLayout(2, 0, [-1, -1], 20011)], types="cn", seed=71)
    con = gpu_console(case)
    con.set_params(case.params)
    l0, m0 = con.forward_loss(with_mix=True)
    l0, m0 = l0.clone(), m0[0].clone()
    con.backward()
    g0 = con.get_grads().clone()
    for phase in ("forward", "backward"):
        if phase == "backward":
            con.forward_loss()
        con.debug_chain_hold(True)
        if phase == "forward":
            con.forward_loss()
        else:
            con.backward()
        torch.cuda.synchronize()
        with pytest.raises(M.MgError) as e:
            con.forward_loss()
        assert e.value.status == M.MG_ERR_TIMEOUT
        con.debug_chain_hold(False)
        l1, m1 = con.forward_loss(with_mix=True)
        con.backward()
        torch.cuda.synchronize()
        assert torch.equal(l1, l0) and torch.equal(m1[0], m0) and torch.equal(con.get_grads(), g0), phase
    con.close()


def test_tma_staged_scans_equal_plain_loads_bitwise():
    """The compressor / gate chunks staged by TMA (bulk tensor copies into swizzled shared memory) and read by
    plain global loads (MG_DYN_TMA=0 at console creation) give bitwise the same mixes, losses and gradients: the
    same values enter the same arithmetic in the same order.  Ragged lengths, several chunks per node, a batch."""
    import os
    import torch
    lays = [W.SongLayout(3, 1, [0, 0, -1], 20011), W.SongLayout(2, 0, [-1, -1], 9001)]
    case = make_case(lays, types="ecng", seed=29)
    cons = []
    old = os.environ.get("MG_DYN_TMA")
    try:
        for flag in ("1", "0"):
            os.environ["MG_DYN_TMA"] = flag
            cons.append(gpu_console(case))
    finally:
        if old is None:
            os.environ.pop("MG_DYN_TMA", None)
        else:
            os.environ["MG_DYN_TMA"] = old
    res = []
    for con in cons:
        con.set_params(case.params)
        con.set_alpha_p(1e-3)
        losses, mixes = con.forward_loss(with_mix=True)
        con.backward()
        res.append((losses.clone(), [m.clone() for m in mixes], con.get_grads().clone()))
    (la, ma, ga), (lb, mb, gb) = res
    assert torch.equal(la, lb) and all(torch.equal(x, y) for x, y in zip(ma, mb)) and torch.equal(ga, gb)
    for con in cons:
        con.close()
