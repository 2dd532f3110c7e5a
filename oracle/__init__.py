"""FP64 CPU oracle for one frictional-contact simulation step and its implicit derivatives.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import or run anything in this package; the library itself never does.  It shares
no code with the CUDA path (``paper_2409_07107_gb300/csrc``) and imports nothing from it.

Everything is plain NumPy, written for clarity, not speed: textbook recursive rigid-body algorithms
in body coordinates (``rigid``), the contact geometry (``contact``), the Coulomb-cone NCP and its
ADMM solve (``ncp``), and the implicit derivatives by two independent routes (``implicit``);
collision detection between convex shapes with App. C's contact-placement terms (``collision``) and
a step with contacts between two bodies built on it (``pair_step``).  Every
function is written so that it also accepts complex arrays: partial derivatives are taken by the
complex-step method (Squire & Trapp 1998), which gives them to machine precision without any
hand-derived derivative formula.
"""
