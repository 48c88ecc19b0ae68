"""Experiment beside the parity tests (not collected by pytest, not part of the library):
per-level TTC/FOE error against ground truth on the 1080p tilted-plane video (the
benchmark's scene, seed 1) for three readings of the Sec. V-B down-sampling:
  A: 2x2 block mean (the oracle's reading)
  B: 2x2 block mean, then a [1 2 1]/4 separable binomial low-pass at the new level
  C: [1 2 1]/4 binomial low-pass, then 2x2 block mean (filter before decimation)
Every level goes through the oracle's own derivative, sum and solve functions; only the
pyramid differs.  Usage: python tests/downsampling_readings.py [pairs] [frame step]."""
import sys, os, json
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np
import oracle, scenes

def blur121(img):
    k = np.array([0.25, 0.5, 0.25])
    p = np.pad(img, 1, mode="edge")
    h = k[0] * p[:, :-2] + k[1] * p[:, 1:-1] + k[2] * p[:, 2:]
    v = k[0] * h[:-2, :] + k[1] * h[1:-1, :] + k[2] * h[2:, :]
    return v

def mean2(img):
    H, W = img.shape
    return img[:H // 2 * 2, :W // 2 * 2].reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))

def pyramid(img, levels, reading):
    out = [img]
    for _ in range(levels - 1):
        x = out[-1]
        if reading == "A":
            x = mean2(x)
        elif reading == "B":
            x = blur121(mean2(x))
        else:
            x = mean2(blur121(x))
        out.append(x)
    return out

def level_results(E0, E1, levels, reading, H, W):
    p0, p1 = pyramid(E0, levels, reading), pyramid(E1, levels, reading)
    recs = []
    for l in range(levels):
        Ex, Ey, Et = oracle.derivatives(p0[l], p1[l])
        pl = 2.0 ** l
        cx = (W - pl) / (2 * pl)
        cy = (H - pl) / (2 * pl)
        s, _ = oracle.sums(Ex, Ey, Et, cx, cy)
        recs.append(oracle.solve(s, 1, l))
    return np.array(recs, dtype=oracle.RESULT_DTYPE)

def main():
    H, W, L = 1080, 1920, 5
    npairs = int(sys.argv[1]) if len(sys.argv) > 1 else 24
    step = int(sys.argv[2]) if len(sys.argv) > 2 else 12
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=1)       # the bench's video (rank 0 seed)
    ts = list(range(0, 299, step))[:npairs]
    out = {}
    for reading in ("A", "B", "C"):
        err_t, err_f = [[] for _ in range(L)], [[] for _ in range(L)]
        rule = {0: ([], []), 1: ([], [])}
        for t in ts:
            fr = scenes.render_sequence(sc, 2, t0=float(t)).numpy().astype(np.float64)
            gt = scenes.ground_truth(sc, t + 0.5)
            r = level_results(fr[0], fr[1], L, reading, H, W)
            for l in range(L):
                err_t[l].append((r[l]["ttc"] - gt[0]) ** 2)
                err_f[l].append((r[l]["x0"] - gt[1]) ** 2 + (r[l]["y0"] - gt[2]) ** 2)
            for ru in (0, 1):
                c = oracle.select_level(r, ru)
                rule[ru][0].append((r[c]["ttc"] - gt[0]) ** 2 if c >= 0 else np.nan)
                rule[ru][1].append(c)
        out[reading] = {"ttc_mse_per_level": [float(np.mean(e)) for e in err_t],
                        "foe_mse_px2_per_level": [float(np.mean(e)) for e in err_f],
                        "ttc_mse_rule0": float(np.nanmean(rule[0][0])), "ttc_mse_rule1": float(np.nanmean(rule[1][0])),
                        "levels_rule0": np.bincount([c for c in rule[0][1] if c >= 0], minlength=L).tolist(),
                        "levels_rule1": np.bincount([c for c in rule[1][1] if c >= 0], minlength=L).tolist()}
        print(reading, json.dumps(out[reading]), flush=True)
    print(json.dumps({"pairs": len(ts), "t": ts, "results": out}))

if __name__ == "__main__":
    main()
