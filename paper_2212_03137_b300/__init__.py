"""B300 (sm_103a) RPMD / adQTB time step behind a C ABI (``include/qhp.h``).

``qhp`` is the ctypes binding of ``libqhp.so``; ``workloads`` generates the
seeded synthetic water boxes; ``build`` compiles the library in-tree.
Importing the package loads nothing: the library is opened on first use.
"""
