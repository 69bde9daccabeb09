"""Training steps fed from pinned host memory, with the host<->device copies
overlapped with the compute of neighbouring steps.

A step takes, per scene, the vertex positions, SDF values and colours, and
for the whole batch the upstream gradients dL/d{image, alpha, depth[,
normal]}, from host memory; it runs pre-filter + forward + backward
(``Rasterizer.step``) and returns dL/dV, dL/df, dL/drgb of every scene to
host memory.  Step i's input copy runs on one stream, its compute on the
caller's stream and its output copy on a third, and two device buffer sets
alternate between steps.  So while step i computes, the copy engines bring
in step i+1's inputs and write out step i-1's gradients.  Every step
computes on its own inputs; events order each buffer's reuse after the step
and the copies that last used it.
"""

from __future__ import annotations

from typing import Sequence

import torch

from .rasterizer import Rasterizer, SceneTensors


class HostStepPipeline:
    """Overlapped host-fed training steps on a sized ``Rasterizer`` (its
    capacities set, e.g. by ``forward()`` + ``shrink_to_fit``).  The scene
    tensors of ``rast`` provide the tet indices; the vertex arrays of every
    step come from the host."""

    def __init__(self, rast: Rasterizer, reduce_grads=None):
        """``reduce_grads``: called with each step's device gradients (per
        scene (dV, df, drgb)) on the compute stream after the backward and
        before they are copied out, e.g. a sum over ranks."""
        self.r = rast
        self.reduce_grads = reduce_grads
        dev = rast.device
        P = rast.total_pixels
        n_up = 4 if rast.params.normals else 3
        self.sets = []
        for _ in range(2):
            scenes = [SceneTensors(torch.empty_like(s.V), s.T, torch.empty_like(s.f),
                                   torch.empty_like(s.rgb)) for s in rast.scenes]
            up = [torch.empty(3 * P, dtype=torch.float32, device=dev),
                  torch.empty(P, dtype=torch.float32, device=dev),
                  torch.empty(P, dtype=torch.float32, device=dev)]
            if n_up == 4:
                up.append(torch.empty(3 * P, dtype=torch.float32, device=dev))
            grads = [(torch.empty_like(s.V), torch.empty_like(s.f), torch.empty_like(s.rgb))
                     for s in rast.scenes]
            self.sets.append((scenes, up, grads))
        self.out = rast._outputs()
        self.h2d = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]
        self.ev_comp = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]
        self.used = [False, False]
        self.i = 0

    def begin(self):
        """Order the copy streams after the work enqueued so far on the
        caller's stream (for example a timing event)."""
        cs = torch.cuda.current_stream(self.r.device)
        self.h2d.wait_stream(cs)
        self.d2h.wait_stream(cs)

    def step(self, host_scenes: Sequence, host_upstream: Sequence, host_grads: Sequence):
        """Enqueue one step.  ``host_scenes``: per scene (V, f, rgb), pinned
        CPU tensors shaped like the rasterizer's scene tensors;
        ``host_upstream``: (dimage, dalpha, ddepth[, dnormal]) flat pinned
        CPU tensors; ``host_grads``: per scene (dV, df, drgb) pinned CPU
        tensors that receive this step's gradients.  Returns the event after
        which those gradients are in host memory.  The host tensors must stay
        unchanged (inputs) and unread (outputs) until then."""
        b = self.i & 1
        scenes, up, grads = self.sets[b]
        cs = torch.cuda.current_stream(self.r.device)
        if self.used[b]:
            self.h2d.wait_event(self.ev_comp[b])     # step i-2 has consumed set b's inputs
        with torch.cuda.stream(self.h2d):
            for d, h in zip(scenes, host_scenes):
                d.V.copy_(h[0], non_blocking=True)
                d.f.copy_(h[1], non_blocking=True)
                d.rgb.copy_(h[2], non_blocking=True)
            for d, h in zip(up, host_upstream):
                d.copy_(h, non_blocking=True)
            self.ev_in[b].record(self.h2d)
        cs.wait_event(self.ev_in[b])
        if self.used[b]:
            cs.wait_event(self.ev_out[b])            # step i-2's gradients have left set b
        self.r.set_scenes(scenes)
        self.r.step(self.out, up, grads)
        if self.reduce_grads is not None:
            self.reduce_grads(grads)
        self.ev_comp[b].record(cs)
        self.d2h.wait_event(self.ev_comp[b])
        with torch.cuda.stream(self.d2h):
            for d, h in zip(grads, host_grads):
                h[0].copy_(d[0], non_blocking=True)
                h[1].copy_(d[1], non_blocking=True)
                h[2].copy_(d[2], non_blocking=True)
            self.ev_out[b].record(self.d2h)
        self.used[b] = True
        self.i += 1
        return self.ev_out[b]

    def end(self):
        """Make the caller's stream wait for every enqueued step's output
        copy."""
        cs = torch.cuda.current_stream(self.r.device)
        for b in range(2):
            if self.used[b]:
                cs.wait_event(self.ev_out[b])
