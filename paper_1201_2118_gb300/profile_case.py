"""A small, fixed workload for profiler captures and timings of the Jacobi
sweep variants.

    python -m paper_1201_2118_gb300.profile_case --n 384 --jacobi 1,4,16,16,4 --sweeps 8
    python -m paper_1201_2118_gb300.profile_case --n 512 --time --sweeps 40 \\
        --jacobi 1,4,16,16,4 7,4,16,64,8 0,4,4,32,4

builds an n^3 lid-driven cavity grid (seeded cavity noise), and for each
given Jacobi variant (kind,vx,ty,zc,stages) runs the requested number of
sweeps on the grid's stream, then checks the device error flag.  With
--stages N it runs N RHS + stage-2 combines per stencil variant
(ty,zc,tile_tz) instead (--order 2 or 4, --form advective or flux).  With
--descriptor N it times N projections u = w - c dt G p by the library's
kernel and by the kernel generated from the equivalent descriptor.  With
--vcycles N it runs N multigrid V-cycles (V(2,2), all levels) on the
pressure equation with R = D U / 1e-3 from the cavity noise, the fine level
smoothed by the first --jacobi variant (default: the grid's).  With
--time, each variant first runs 4 warm-up sweeps and the timed sweeps are
bracketed by CUDA events on the grid's stream; the line printed per variant
gives microseconds per sweep and the algorithmic bytes (read p and r, write
p) per second.  With --blocks the grid is the 64-block workload instead
(per-axis widths U{16..96}, seed 2, periodic, curl-noise start; ghost width
1 with --order 2, 2 with --order 4).  With --ghost N it runs N ghost fills
of each array list given by --arrays (e.g. p r,p u,v,w,p).  The launch to
capture under ncu is selected with -k/-s/-c.

    python -m paper_1201_2118_gb300.profile_case --blocks --order 4 --ghost 5 --arrays p r,p u,v,w,p
    python -m paper_1201_2118_gb300.profile_case --blocks --order 4 --time --sweeps 20 \\
        --jacobi 9,2,8,32,6 7,2,8,32,6
"""
import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=384)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--jacobi", nargs="*", default=[], help="kind,vx,ty,zc,stages ...")
    ap.add_argument("--sweeps", type=int, default=12)
    ap.add_argument("--time", action="store_true")
    ap.add_argument("--stages", type=int, default=0,
                    help="instead of sweeps: this many RHS + stage-2 combines per stencil variant")
    ap.add_argument("--stencil", nargs="*", default=[], help="ty,zc,tile_tz ...")
    ap.add_argument("--order", type=int, default=2, choices=[2, 4])
    ap.add_argument("--form", default="advective", choices=["advective", "flux"])
    ap.add_argument("--vcycles", type=int, default=0,
                    help="instead of sweeps: this many multigrid V-cycles")
    ap.add_argument("--descriptor", type=int, default=0,
                    help="instead of sweeps: this many projections by the library's kernel "
                         "and by the same projection generated from a kernel descriptor")
    ap.add_argument("--blocks", action="store_true",
                    help="the 64-block workload instead of the n^3 cavity")
    ap.add_argument("--ghost", type=int, default=0,
                    help="instead of sweeps: this many ghost fills of each --arrays list")
    ap.add_argument("--arrays", nargs="*", default=["p"], help="array lists, e.g. p r,p u,v,w,p")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import workloads
    from paper_1201_2118_gb300 import Grid
    n = a.n
    s = torch.cuda.Stream()
    if a.blocks:
        cfg = workloads.WORKLOADS["blocks64"]
        gd, blocks = workloads.block_tiling(seed=cfg["tiling_seed"])
        h = workloads.workload_h("blocks64")
        g = Grid(ghost=1 if a.order == 2 else 2, h=h, dtype=a.dtype, stream=s,
                 blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
        g.set_params(cfg["nu"], cfg["jacobi_iters"], 1.0, a.order)
        g.set_advection(a.form)
        g.upload_blocks(workloads.split_blocks(workloads.random_div_free(gd, h, seed=cfg["ic_seed"]),
                                               blocks))
        cells = gd[0] * gd[1] * gd[2]
        name = "blocks64 g=%d" % (1 if a.order == 2 else 2)
    else:
        g = Grid((n, n, n), ghost=1 if a.order == 2 else 2, h=(1.0 / n,) * 3, dtype=a.dtype,
                 stream=s)
        g.set_cavity(1.0)
        g.set_params(1e-3, 50, 1.0, a.order)
        g.set_advection(a.form)
        g.upload(workloads.ldc_noise(n, seed=1))
        cells = n ** 3
        name = "%d^3" % n
    g.pressure_solve(1e-3, 0)
    es = 4 if a.dtype == "f32" else 2
    if a.ghost:
        import paper_1201_2118_gb300 as pk
        for lst in a.arrays:
            m = pk.mask(*[getattr(pk, x.strip().upper()) for x in lst.split(",")])
            if a.time:
                g.ghost_fill(m)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
            for _ in range(a.ghost):
                g.ghost_fill(m)
            if a.time:
                e1.record(s)
            torch.cuda.synchronize()
            print("%s %s ghost fill of %s%s" % (name, a.dtype, lst, " %.1f us" % (
                e0.elapsed_time(e1) * 1e3 / a.ghost) if a.time else ""), flush=True)
        g.check()
        return
    if a.descriptor:
        from paper_1201_2118_gb300 import (Descriptor, GeneratedKernel, P, SET_U1, U1, V1, W1, WU,
                                           WV, WW)
        d = Descriptor(
            name="update_velocity", inputs={"wu": "cached", "wv": "cached", "ww": "cached",
                                            "p": "cached"},
            outputs=["u", "v", "w"], params=["cdt"], stencil=(0, 1, 0, 1, 0, 1),
            body='''
              const float pc = at(p, 0, 0, 0);
              out(u) = at(wu, 0, 0, 0) - cdt * ((at(p, 1, 0, 0) - pc) * idx);
              out(v) = at(wv, 0, 0, 0) - cdt * ((at(p, 0, 1, 0) - pc) * idy);
              out(w) = at(ww, 0, 0, 0) - cdt * ((at(p, 0, 0, 1) - pc) * idz);
            ''')
        kern = GeneratedKernel(d)
        d_direct = Descriptor(name="update_velocity_direct",
                              inputs={v: "direct" for v in d.inputs}, outputs=d.outputs,
                              params=d.params, stencil=d.stencil, body=d.body)
        kern_direct = GeneratedKernel(d_direct)
        bind = {"wu": WU, "wv": WV, "ww": WW, "p": P, "u": U1, "v": V1, "w": W1}
        runs = {"library cfd_project (kernel + ghost fill of the output)":
                    lambda: g.project(1e-3, SET_U1),
                "generated, inputs cached in the plane ring": lambda: kern(g, bind, cdt=1e-3),
                "generated, inputs read directly": lambda: kern_direct(g, bind, cdt=1e-3)}
        for name, fn in runs.items():
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(a.descriptor):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / a.descriptor
            gbs = 7 * es * n ** 3 / (us * 1e-6) / 1e9  # read w (3), p; write u (3)
            print("%d^3 projection, %s: %.1f us %.0f GB/s" % (n, name, us, gbs), flush=True)
        g.check()
        return
    if a.vcycles:
        from paper_1201_2118_gb300 import P, U, V, W, WU, WV, WW, mask
        if a.jacobi:
            g.set_kernel_config(jacobi=tuple(int(x) for x in a.jacobi[0].split(",")))
        with torch.cuda.stream(s):
            for x, y in ((U, WU), (V, WV), (W, WW)):
                g.interior(y).copy_(g.interior(x))
            g.interior(P).zero_()
        g.ghost_fill(mask(WU, WV, WW, P))
        g.pressure_solve(1e-3, 0)
        g.mg_vcycles(1)  # captures the cycle's graph
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.mg_vcycles(a.vcycles)
        e1.record(s)
        torch.cuda.synchronize()
        print("%d^3 %s jacobi %s levels %d: %.3f ms per V-cycle" %
              (n, a.dtype, g.kernel_config()[0], g.multigrid_levels(),
               e0.elapsed_time(e1) / a.vcycles), flush=True)
        g.check()
        return
    if a.stages:
        from paper_1201_2118_gb300 import SET_U, SET_U1, SET_W
        for c in a.stencil or [None]:
            if c is not None:
                g.set_kernel_config(stencil=tuple(int(x) for x in c.split(",")))
            cfg = g.kernel_config()[1]
            # stage-2 form: w = 1/2 u + 1/2 u1 + 1/2 dt F(u1), 36 B/cell
            run = lambda k: [g.stage(0.5, SET_U, 0.5, SET_U1, 1e-4, SET_W) for _ in range(k)]
            if not a.time:
                run(a.stages)
                torch.cuda.synchronize()
                print("ok", n, a.dtype, "stencil", cfg, a.stages, flush=True)
                continue
            run(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            run(a.stages)
            e1.record(s)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / a.stages
            gbs = 9 * es * n ** 3 / (us * 1e-6) / 1e9
            print("%d^3 %s order %d %s stencil %s %.1f us/stage %.0f GB/s" %
                  (n, a.dtype, a.order, a.form, cfg, us, gbs), flush=True)
        g.check()
        return
    for c in a.jacobi or [None]:
        if c is not None:
            g.set_kernel_config(jacobi=tuple(int(x) for x in c.split(",")))
        cfg = g.kernel_config()[0]
        if not a.time:
            g.jacobi(a.sweeps)
            torch.cuda.synchronize()
            print("ok", name, a.dtype, cfg, a.sweeps, flush=True)
            continue
        g.jacobi(4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.jacobi(a.sweeps)
        e1.record(s)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / a.sweeps
        gbs = 3 * es * cells / (us * 1e-6) / 1e9
        print("%s %s %s %.1f us/sweep %.0f GB/s" % (name, a.dtype, cfg, us, gbs), flush=True)
    g.check()


if __name__ == "__main__":
    main()
