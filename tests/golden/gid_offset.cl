__kernel void gid(__global int *data)
{
    data[get_global_id(0)] = (int)get_global_id(0);
}
