"""Plain-form baseline: a per-subdomain loop of eager PyTorch autograd.

This is how the method is usually written (and how the paper's own pipeline
computes it before CUDA-graph capture, Sec. 2.3): every subdomain net is an
ordinary MLP, the derivatives for the Navier-Stokes residuals come from
``torch.autograd.grad(..., create_graph=True)``, the loss is assembled per net
(Eq. (16)) and ``loss.backward()`` runs the double backward; the optimiser is
``torch.optim.Adam``.

It is *not* the oracle and not the product: the benchmark times it on the GPU
in FP32 as the comparison arm, and the CPU tests run it in FP64 as an
independent library cross-check of the oracle's hand-written reverse pass.
It uses the same readings as the oracle: inputs mapped from each net's box to
[-1, 1], shared face points as the ghost set, anchor normalisation on the
pressure a master sends (Eq. (15)), lambda^space = 0 on masters.
"""
from __future__ import annotations

import math

import torch


class PlainForm:
    def __init__(self, problem, device="cpu", dtype=torch.float32, theta=None):
        import numpy as np
        from paper_2602_15883_b300 import synth

        cfg = problem.cfg
        self.cfg = cfg
        self.dev, self.dt = torch.device(device), dtype
        self.ds = cfg["d_space"]
        self.din = synth.d_in(cfg)
        self.dout = synth.d_out(cfg)
        self.unst = cfg["unsteady"]
        self.nn = synth.n_nets(cfg)
        self.npar = synth.n_params_net(cfg)
        self.shapes = synth.layer_shapes(cfg)
        self.faces = synth.faces(cfg)
        th = problem.theta0 if theta is None else theta
        th = torch.as_tensor(np.asarray(th, np.float64), dtype=dtype, device=self.dev)
        self.params = []
        for k in range(self.nn):
            blk, off, ps = th[k * self.npar:(k + 1) * self.npar], 0, []
            for (o, i) in self.shapes:
                W = blk[off:off + o * i].reshape(o, i).clone().requires_grad_(True); off += o * i
                b = blk[off:off + o].clone().requires_grad_(True); off += o
                ps += [W, b]
            self.params.append(ps)
        self.center, self.scale = [], []
        for k in range(self.nn):
            lo, hi = synth.net_box(cfg, k)
            self.center.append(torch.tensor(0.5 * (lo + hi), dtype=dtype, device=self.dev))
            self.scale.append(torch.tensor(2.0 / (hi - lo), dtype=dtype, device=self.dev))
        # master flags (anchor's spatial cell, FP32 cell rule)
        acell = [self._cell(a, cfg["anchor"][a]) for a in range(self.ds)]
        self.master = []
        for k in range(self.nn):
            c = synth.cell_of_net(cfg, k)
            self.master.append(all(c[a] == acell[a] for a in range(self.ds)))
        t = lambda a: torch.as_tensor(np.asarray(a), device=self.dev)
        ro = np.concatenate([[0], np.cumsum(problem.res_counts)])
        oo = np.concatenate([[0], np.cumsum(problem.obs_counts)])
        fo = np.concatenate([[0], np.cumsum(problem.face_counts)])
        self.res = [t(problem.res_pts[ro[k]:ro[k + 1]]).to(dtype) for k in range(self.nn)]
        self.obs = [t(problem.obs_pts[oo[k]:oo[k + 1]]).to(dtype) for k in range(self.nn)]
        self.obsv = [t(problem.obs_vals[oo[k]:oo[k + 1]]).to(dtype) for k in range(self.nn)]
        self.fpts = [t(problem.face_pts[fo[f]:fo[f + 1]]).to(dtype) for f in range(len(self.faces))]
        self.net_faces = [[] for _ in range(self.nn)]
        for f, (a, b, ax) in enumerate(self.faces):
            self.net_faces[a].append((f, 0))
            self.net_faces[b].append((f, 1))
        self.w = torch.tensor(cfg["comp_w"][: self.ds], dtype=dtype, device=self.dev)
        # volumetric ghost layers: per net, its ghost points grouped by owner
        self.ghost = None
        if getattr(problem, "ghost_counts", None) is not None:
            go = np.concatenate([[0], np.cumsum(problem.ghost_counts)])
            owners = synth.owner_net(cfg, problem.ghost_pts)
            self.ghost = []
            for k in range(self.nn):
                own = owners[go[k]:go[k + 1]]
                pts = problem.ghost_pts[go[k]:go[k + 1]]
                groups = []
                for B in sorted(set(own.tolist())):
                    same_space = all(synth.cell_of_net(cfg, k)[a] == synth.cell_of_net(cfg, B)[a]
                                     for a in range(self.ds))
                    groups.append((B, t(pts[own == B]).to(dtype), bool(self.unst and same_space)))
                self.ghost.append(groups)
        self.opt = torch.optim.Adam([p for ps in self.params for p in ps], lr=cfg["lr"],
                                    betas=(cfg["beta1"], cfg["beta2"]), eps=cfg["eps"])
        iv = int(cfg.get("lr_decay_interval", 0))
        self.sched = (torch.optim.lr_scheduler.StepLR(self.opt, step_size=iv, gamma=cfg.get("lr_decay_factor", 1.0))
                      if iv > 0 else None)
        self.comm_interval = int(cfg.get("comm_interval", 1))
        self.t = 0
        self.msgs = None
        self.anchor_t = torch.tensor(np.float32(cfg["anchor"][: self.ds]), dtype=dtype, device=self.dev)
        self.graph = None

    def _cell(self, a, x):
        import numpy as np
        lo, hi = np.float32(self.cfg["lo"][a]), np.float32(self.cfg["hi"][a])
        inv_h = np.float32(self.cfg["splits"][a] / (self.cfg["hi"][a] - self.cfg["lo"][a]))
        q = np.float32(np.float32(np.float32(x) - lo) * inv_h)
        return int(min(max(math.floor(q), 0), self.cfg["splits"][a] - 1))

    # ------------------------------------------------------------------
    def net(self, k, x):
        h = (x - self.center[k]) * self.scale[k]
        ps = self.params[k]
        nl = len(ps) // 2
        for l in range(nl):
            h = torch.nn.functional.linear(h, ps[2 * l], ps[2 * l + 1])
            if l < nl - 1:
                h = torch.sin(h) if self.cfg.get("activation", 0) == 1 else torch.tanh(h)
        return h

    def residual(self, k, x):
        x = x.detach().requires_grad_(True)
        y = self.net(k, x)
        ds = self.ds
        grads = [torch.autograd.grad(y[:, j].sum(), x, create_graph=True)[0] for j in range(self.dout)]
        r = []
        for j in range(ds):
            lap = 0.0
            for s in range(ds):
                lap = lap + torch.autograd.grad(grads[j][:, s].sum(), x, create_graph=True)[0][:, s]
            v = sum(y[:, i] * grads[j][:, i] for i in range(ds)) + grads[ds][:, j] - self.cfg["nu"] * lap
            if self.unst:
                v = v + grads[j][:, ds]
            r.append(v)
        r.append(sum(grads[i][:, i] for i in range(ds)))
        return torch.stack(r, 1)

    def _message(self, k, x):
        """Net k's velocity and (anchor-normalised if k is a master) pressure at x."""
        y = self.net(k, x)
        P = y[:, self.ds]
        if self.master[k]:
            import numpy as np
            xa = x.clone()
            xa[:, : self.ds] = self.anchor_t
            P = P - self.net(k, xa)[:, self.ds]
        return y[:, : self.ds], P

    def exchange(self):
        """Neighbour messages at the current parameters (detached)."""
        import numpy as np
        if self.ghost is not None:
            with torch.no_grad():
                return [[(B, x, tm, self._message(B, x)) for (B, x, tm) in groups] for groups in self.ghost]
        msgs = []
        with torch.no_grad():
            for f, (a, b, ax) in enumerate(self.faces):
                x = self.fpts[f]
                sides = []
                for k in (a, b):
                    y = self.net(k, x)
                    P = y[:, self.ds]
                    if self.master[k]:
                        xa = x.clone()
                        xa[:, : self.ds] = self.anchor_t
                        P = P - self.net(k, xa)[:, self.ds]
                    sides.append((y[:, : self.ds], P))
                msgs.append(sides)
        return msgs

    def net_losses(self, k, msgs):
        cfg = self.cfg
        z = torch.zeros((), dtype=self.dt, device=self.dev)
        lobs = lpde = lgu = lsp = ltm = z
        if len(self.res[k]):
            lpde = (self.residual(k, self.res[k]) ** 2).sum(1).mean()
        if len(self.obs[k]):
            e = self.net(k, self.obs[k])[:, : self.ds] - self.obsv[k]
            lobs = (self.w * e * e).sum(1).mean()
        if self.ghost is not None:
            ngh = sum(len(x) for (_, x, _) in self.ghost[k])
            for (B, x, tm, (U, P)) in msgs[k]:
                y = self.net(k, x)
                e = y[:, : self.ds] - U
                lgu = lgu + (self.w * e * e).sum() / ngh
                ep = ((y[:, self.ds] - P) ** 2).sum() / ngh
                if tm:
                    ltm = ltm + ep
                else:
                    lsp = lsp + ep
        ngh = sum(len(self.fpts[f]) for f, _ in self.net_faces[k])
        for f, side in (self.net_faces[k] if self.ghost is None else []):
            U, P = msgs[f][1 - side]
            y = self.net(k, self.fpts[f])
            e = y[:, : self.ds] - U
            lgu = lgu + (self.w * e * e).sum() / ngh
            ep = ((y[:, self.ds] - P) ** 2).sum() / ngh
            if self.unst and self.faces[f][2] == self.ds:
                ltm = ltm + ep
            else:
                lsp = lsp + ep
        lam_sp = 0.0 if self.master[k] else cfg["lambda_gh_p_space"]
        total = (cfg["lambda_obs"] * lobs + cfg["lambda_pde"] * lpde + cfg["lambda_gh_u"] * lgu
                 + lam_sp * lsp + cfg["lambda_gh_p_time"] * ltm)
        return torch.stack([lobs, lpde, lgu, lsp, ltm, total])

    def losses_and_grads(self):
        # Algorithm 1: messages refreshed every I_comm iterations, reused between
        if self.msgs is None or self.t % self.comm_interval == 0:
            self.msgs = self.exchange()
        msgs = self.msgs
        recs = []
        for k in range(self.nn):
            for p in self.params[k]:
                p.grad = None
            rec = self.net_losses(k, msgs)
            rec[5].backward()
            recs.append(rec.detach())
        return torch.stack(recs)

    def step(self):
        rec = self.losses_and_grads()
        clip = self.cfg["clip_norm"]
        if clip > 0:
            for k in range(self.nn):
                torch.nn.utils.clip_grad_norm_(self.params[k], clip)
        self.opt.step()
        if self.sched is not None:
            self.sched.step()
        self.t += 1
        return rec

    def capture(self, warmup=3):
        """Capture one whole training step (exchange, per-net losses, double
        backward, Adam) in a CUDA graph, the way the paper's pipeline replays
        its step (Sec. 2.3); then ``replay()`` runs a step.  Needs a CUDA
        device, I_comm = 1, no learning-rate schedule and no clipping."""
        if self.dev.type != "cuda" or self.comm_interval != 1 or self.sched is not None or self.cfg["clip_norm"] > 0:
            raise ValueError("graph capture needs CUDA, I_comm = 1, no LR schedule and no clipping")
        params = [p for ps in self.params for p in ps]
        self.opt = torch.optim.Adam(params, lr=self.cfg["lr"], betas=(self.cfg["beta1"], self.cfg["beta2"]),
                                    eps=self.cfg["eps"], capturable=True)
        snap = [p.detach().clone() for p in params]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.msgs = None
                self.losses_and_grads()
                self.opt.step()
        torch.cuda.current_stream().wait_stream(side)
        # the warm-up steps are undone: parameters and Adam state as before
        with torch.no_grad():
            for p, p0 in zip(params, snap):
                p.copy_(p0)
            for st in self.opt.state.values():
                for v in st.values():
                    if torch.is_tensor(v):
                        v.zero_()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.msgs = None
            self.rec_static = self.losses_and_grads()
            self.opt.step()
        return self

    def replay(self):
        self.graph.replay()
        self.t += 1
        return self.rec_static

    def flat(self, grads=False):
        out = []
        for ps in self.params:
            for p in ps:
                t = p.grad if grads else p
                out.append((t if t is not None else torch.zeros_like(p)).detach().reshape(-1))
        return torch.cat(out)
