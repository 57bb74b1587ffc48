"""The library's host planner against the oracle, on the CPU.

The planner (csrc/geometry.cpp: tree, partition into cells, edges and faces,
near fields, column groups) runs on the host in the GPU path; here it is
compiled with a small harness (tests/plan_replay.cpp) and fed the oracle's own
skeletonization decisions sublevel by sublevel, so that every plan can be
compared with the oracle's index sets box by box: the root box and depth
(Sec. 3.1 / 4.1), the sublevel sequence (Algorithms 4.1 / 4.2), and per box
its DOFs, its near field (the proxy interior and the SCI-coupled DOFs,
Sec. 3.3 / 4.3) and its column groups (Sec. 4.4, Lemma 4.2).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import hif_inputs as hi
from oracle import hifie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KIND = {"cell": 0, "face": 1, "edge": 2}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("replay") / "plan_replay"
    subprocess.run([gxx, "-O1", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-o", str(out),
                    os.path.join(ROOT, "tests", "plan_replay.cpp"),
                    os.path.join(ROOT, "paper_1307_2666_gb300", "csrc", "geometry.cpp")], check=True)
    return str(out)


def _replay(harness, pb, eps, c=None, occupancy=64, second_kind=True):
    c = pb.c if c is None else c
    sets = []
    hifie.factor(pb.points, pb.weights, pb.a, pb.b, c, pb.kernel_id, eps, pb.proxy, occupancy=occupancy,
                 second_kind=second_kind, trace_sets=sets)
    subs = []                                   # the oracle's boxes, sublevel by sublevel
    for e in sets:
        if not subs or subs[-1][0] != (e[0], e[1]):
            subs.append(((e[0], e[1]), []))
        subs[-1][1].append(e)
    N, d = pb.points.shape
    lines = [f"{N} {d} {occupancy} 1.5 {1 if second_kind else 0}", " ".join(repr(float(v)) for v in pb.points.reshape(-1)),
             " ".join(repr(float(v)) for v in pb.weights), str(len(subs))]
    for _, boxes in subs:
        lines.append(str(len(boxes)))
        for e in boxes:
            sk, rd = e[5], e[6]
            lines.append(" ".join(map(str, [sk.size, *sk.tolist(), rd.size, *rd.tolist()])))
    r = subprocess.run([harness], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return subs, r.stdout.split("\n")


def _parse(out):
    tree = plan = None
    subs = []
    it = iter(out)
    for ln in it:
        f = ln.split()
        if not f:
            continue
        if f[0] == "TREE":
            tree = (np.array([float(v) for v in f[1:4]]), float(f[4]), int(f[5]))
        elif f[0] == "PLAN":
            v = list(map(int, f[1:]))
            plan = list(zip(v[0::2], v[1::2]))
        elif f[0] == "SUB":
            subs.append(((int(f[1]), int(f[2])), []))
        elif f[0] == "BOX":
            mem = np.array(next(it).split()[2:], dtype=np.int64)
            near = np.array(next(it).split()[2:], dtype=np.int64)
            ng = int(next(it).split()[1])
            groups = []
            for _ in range(ng):
                g = next(it).split()
                groups.append(np.array(g[3:], dtype=np.int64))
            subs[-1][1].append((mem, near, groups))
    return tree, plan, subs


@pytest.mark.parametrize("case", ["2d-symmetric", "2d-b-ne-c-ragged", "2d-n64", "2d-odd-cells", "2d-no-groups",
                                  "2d-jittered", "3d", "3d-occ27", "3d-n16"])
def test_host_plan_matches_oracle_sets(harness, case):
    occ, second_kind = 64, True
    if case == "2d-symmetric":
        pb, c, eps = hi.volume_problem(32, 2, smooth_seed=21), None, 1e-6
    elif case == "2d-b-ne-c-ragged":
        pb = hi.volume_problem(48, 2, smooth_seed=22)
        c, eps = pb.c * (1.0 + 0.5 * hi.smooth_field(pb.points, 23)), 1e-6
    elif case == "2d-n64":
        pb, c, eps = hi.volume_problem(64, 2, smooth_seed=1002), None, 1e-6
    elif case == "2d-odd-cells":
        # 5 x 5 DOFs per leaf cell: DOFs lie exactly on the proxy circles of the edges
        pb, c, eps = hi.volume_problem(40, 2, smooth_seed=26), None, 1e-6
    elif case == "2d-no-groups":
        # without the Sec. 4.4 modifications: one group per box
        pb, c, eps, second_kind = hi.volume_problem(32, 2, smooth_seed=27), None, 1e-6, False
    elif case == "2d-jittered":
        # points off the grid (uniform jitter of up to 0.3 h): no exact ties anywhere
        pb, c, eps = hi.volume_problem(32, 2, smooth_seed=29), None, 1e-6
        pb.points = pb.points + 0.3 / 32 * (np.random.default_rng(29).uniform(size=pb.points.shape) - 0.5)
    elif case == "3d":
        pb, c, eps = hi.volume_problem(12, 3, smooth_seed=24), None, 1e-3
    elif case == "3d-occ27":
        pb, c, eps, occ = hi.volume_problem(12, 3, smooth_seed=5), None, 1e-3, 27
    else:
        pb, c, eps = hi.volume_problem(16, 3, smooth_seed=25), None, 1e-3
    osubs, out = _replay(harness, pb, eps, c, occupancy=occ, second_kind=second_kind)
    tree, plan, csubs = _parse(out)
    # tree and sublevel sequence
    lo, W = hifie.root_box(pb.points, pb.weights)
    L = hifie.num_levels(pb.points, lo, W, occ)
    d = pb.points.shape[1]
    np.testing.assert_allclose(tree[0][:d], lo, rtol=0, atol=1e-15)
    assert tree[1] == pytest.approx(W, rel=1e-15) and tree[2] == L
    assert plan == [(KIND[k], l) for k, l in hifie.sublevel_plan(d, L)]
    # every sublevel's boxes, near fields and groups
    assert [s[0] for s in csubs] == [(KIND[k], l) for (k, l), _ in osubs]
    nbox = ngrp = 0
    for (_, oboxes), (_, cboxes) in zip(osubs, csubs):
        assert len(cboxes) == len(oboxes)
        for o, (mem, near, groups) in zip(oboxes, cboxes):
            np.testing.assert_array_equal(mem, o[2])
            np.testing.assert_array_equal(near, o[3])
            assert len(groups) == len(o[4])
            for g, og in zip(groups, o[4]):
                np.testing.assert_array_equal(g, og)
            nbox += 1
            ngrp += len(groups)
    # the comparison covered SCI groups, not only single-group boxes
    assert nbox > 20 and (ngrp > nbox if second_kind else ngrp == nbox)


def test_batched_plans_concatenate(tmp_path):
    # a batched handle's sublevel plan is its problems' plans one after the
    # other (append_plan): every array concatenated, the box, near-field and
    # group offsets shifted by what precedes them; 1 to 4 problems, empty
    # near fields included
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "append"
    subprocess.run([gxx, "-O1", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(ROOT, "tests", "plan_append_harness.cpp"),
                    os.path.join(ROOT, "paper_1307_2666_gb300", "csrc", "geometry.cpp")], check=True)
    rng = np.random.default_rng(3)
    for trial in range(40):
        plans = []
        for _ in range(int(rng.integers(1, 5))):
            boxes = []
            for _ in range(int(rng.integers(1, 6))):
                mem = rng.integers(0, 1000, int(rng.integers(1, 6))).tolist()
                near = rng.integers(0, 1000, int(rng.integers(0, 6))).tolist()
                groups = [(int(rng.integers(0, 5)), int(rng.integers(1, 5)), int(rng.integers(0, 2)))
                          for _ in range(int(rng.integers(1, 3)))]
                boxes.append((mem, near, groups, int(rng.integers(0, 2)), rng.standard_normal(3).tolist()))
            plans.append(boxes)
        lines = [str(len(plans))]
        for boxes in plans:
            lines.append(str(len(boxes)))
            for mem, near, groups, sci, ctr in boxes:
                lines.append(" ".join(map(str, [len(mem), *mem, len(near), *near, len(groups)]
                                          + [v for g in groups for v in g] + [sci])) + " " +
                             " ".join(repr(c) for c in ctr))
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        got = {}
        for ln in out:
            f = ln.split()
            if f:
                got[f[0]] = [float(v) for v in f[2:]] if f[0] != "nbox" else int(f[1])
        allb = [b for boxes in plans for b in boxes]
        exp = {"nbox": len(allb), "members": [], "near": [], "grp_col0": [], "grp_n": [], "grp_sci": [],
               "box_sci": [], "centers": [], "box_off": [0], "near_off": [0], "grp_off": [0]}
        for mem, near, groups, sci, ctr in allb:
            exp["members"] += mem
            exp["near"] += near
            exp["grp_col0"] += [g[0] for g in groups]
            exp["grp_n"] += [g[1] for g in groups]
            exp["grp_sci"] += [g[2] for g in groups]
            exp["box_sci"].append(sci)
            exp["centers"] += ctr
            exp["box_off"].append(len(exp["members"]))
            exp["near_off"].append(len(exp["near"]))
            exp["grp_off"].append(len(exp["grp_col0"]))
        exp["cols"] = exp["members"]
        assert got["nbox"] == exp["nbox"]
        for k in exp:
            if k != "nbox":
                assert got[k] == [float(v) for v in exp[k]], (trial, k)


def test_uniform_grid_detection(tmp_path):
    # the direct sum takes the grid convolution (and the tensor-core path)
    # only for points that fill a full uniform n^d grid with cell volumes h^d,
    # in any order; any other point set keeps the general sum
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "grid"
    subprocess.run([gxx, "-O1", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(ROOT, "tests", "grid_layout_harness.cpp"),
                    os.path.join(ROOT, "paper_1307_2666_gb300", "csrc", "geometry.cpp")], check=True)

    def run(pts, w, off=0):
        N, d = pts.shape
        inp = f"{N} {d} {off}\n" + " ".join(repr(float(v)) for v in pts.reshape(-1)) + "\n" + \
            " ".join(repr(float(v)) for v in w) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        if out[0] == "0":
            return None
        return int(out[1]), float(out[2]), np.array(out[3:], dtype=np.int64)

    for n, d in [(8, 2), (5, 3), (2, 2)]:
        pts, w = hi.grid_points(n, d)
        r = run(pts, w, off=100)
        assert r is not None and r[0] == n and r[1] == pytest.approx(1.0 / n, rel=1e-14)
        np.testing.assert_array_equal(r[2], np.arange(n ** d) + 100)      # first coordinate slowest
        perm = np.random.default_rng(n).permutation(n ** d)
        r = run(pts[perm], w[perm])
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        np.testing.assert_array_equal(r[2], inv)                           # grid position -> permuted DOF
    pts, w = hi.grid_points(8, 2)
    h = 1.0 / 8
    assert run(pts[:-1], w[:-1]) is None                                   # a point missing
    p2 = pts.copy()
    p2[5] += 1e-3 * h
    assert run(p2, w) is None                                              # off the grid
    p3 = pts.copy()
    p3[7] = p3[8]
    assert run(p3, w) is None                                              # two points in one cell
    w2 = w.copy()
    w2[3] *= 1.5
    assert run(pts, w2) is None                                            # unequal weights
    assert run(pts, 2.0 * w) is None                                       # weights are not h^d
    p4 = pts.copy()
    p4[:, 0] *= 2.0
    assert run(p4, w) is None                                              # unequal spacing per axis


# planted mistakes in a copy of the planner: the replay must see each one
PLANNER_MUTATIONS = [
    ("proxy-boundary-included", "const double R2 = R * R * (1.0 - kTie);", "const double R2 = R * R * (1.0 + kTie);"),
    ("inactive-sci-neighbours", "if (active[i] && box_of[i] != b && mark[i] != ep) {",
     "if (box_of[i] != b && mark[i] != ep) {"),
    ("upper-edge-candidates-missing", "jhi[k] = std::min(s - 1, c[k] + 2); }",
     "jhi[k] = std::min(s - 1, c[k]); }"),
    ("own-box-in-patterns", "if (active[i] && box_of[i] != b && mark[i] != ep) {",
     "if (active[i] && mark[i] != ep) {"),
    ("ties-to-highest-id", "if (cd2[e] <= lim && (best_id < 0 || cid[e] < best_id)) best_id = cid[e];",
     "if (cd2[e] <= lim && (best_id < 0 || cid[e] > best_id)) best_id = cid[e];"),
]


def test_replay_sees_planted_planner_mistakes(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    import concurrent.futures as cf
    src = open(os.path.join(ROOT, "paper_1307_2666_gb300", "csrc", "geometry.cpp")).read()
    pb = hi.volume_problem(40, 2, smooth_seed=26)          # on-circle DOFs, SCI groups
    c = pb.c * (1.0 + 0.5 * hi.smooth_field(pb.points, 28))

    def build(name, text):
        d = tmp_path / name
        d.mkdir()
        (d / "geometry.cpp").write_text(text)
        exe = d / "replay"
        subprocess.run([gxx, "-O1", "-std=c++17", "-fopenmp", "-ffp-contract=off",
                        "-I", os.path.join(ROOT, "paper_1307_2666_gb300", "csrc"), "-o", str(exe),
                        os.path.join(ROOT, "tests", "plan_replay.cpp"), str(d / "geometry.cpp")], check=True)
        return str(exe)

    def matches(exe):
        try:
            osubs, out = _replay(exe, pb, 1e-6, c)
        except subprocess.CalledProcessError:
            return False                                  # the planted mistake broke the planner outright
        _, _, csubs = _parse(out)
        if [len(s[1]) for s in csubs] != [len(s[1]) for s in osubs]:
            return False
        for (_, oboxes), (_, cboxes) in zip(osubs, csubs):
            for o, (mem, near, groups) in zip(oboxes, cboxes):
                if not (np.array_equal(mem, o[2]) and np.array_equal(near, o[3]) and len(groups) == len(o[4])
                        and all(np.array_equal(g, og) for g, og in zip(groups, o[4]))):
                    return False
        return True

    cases = PLANNER_MUTATIONS
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        exes = {name: ex.submit(build, name, src.replace(old, new, 1)) for name, old, new in cases}
        exes["unplanted"] = ex.submit(build, "unplanted", src)
        exes = {k: f.result() for k, f in exes.items()}
    for name, old, _ in cases:
        assert src.count(old) == 1, name
    assert matches(exes["unplanted"])
    for name, _, _ in cases:
        assert not matches(exes[name]), f"planted planner mistake not seen: {name}"


@pytest.mark.parametrize("seed", range(6))
def test_host_plan_random_configurations(harness, seed):
    # random sizes, occupancies, coefficients and (for some) off-grid points:
    # the planner's sets equal the oracle's for every box
    rng = np.random.default_rng(100 + seed)
    dim = 2 if seed < 4 else 3
    n = int(rng.integers(16, 41)) if dim == 2 else int(rng.integers(6, 11))
    occ = int(rng.choice([16, 27, 64]))
    pb = hi.volume_problem(n, dim, smooth_seed=200 + seed)
    c = pb.c * (1.0 + 0.4 * hi.smooth_field(pb.points, 300 + seed)) if seed % 2 else None
    if seed in (2, 5):
        pb.points = pb.points + 0.2 / n * (rng.uniform(size=pb.points.shape) - 0.5)
    osubs, out = _replay(harness, pb, 1e-4, c, occupancy=occ)
    tree, plan, csubs = _parse(out)
    assert [s[0] for s in csubs] == [(KIND[k], l) for (k, l), _ in osubs]
    for (_, oboxes), (_, cboxes) in zip(osubs, csubs):
        assert len(cboxes) == len(oboxes)
        for o, (mem, near, groups) in zip(oboxes, cboxes):
            np.testing.assert_array_equal(mem, o[2])
            np.testing.assert_array_equal(near, o[3])
            assert len(groups) == len(o[4])
            for g, og in zip(groups, o[4]):
                np.testing.assert_array_equal(g, og)
